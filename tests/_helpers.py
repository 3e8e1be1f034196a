"""Layout helpers shared by the GPU parity tests: the ABI's packed path is the
oracle's (m_0, ..., m_{d-1}, f) flattened in the same [t][c][y][x] order."""
import numpy as np

import oracle as o


def oracle_grid(n, bc, P):
    return o.Grid(tuple(n), tuple("periodic" if b in ("periodic", 0) else "neumann" for b in bc), P)


def pack_path(g, m, f):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in m] + [np.asarray(f, np.float64).ravel()])


def unpack_path(g, vec):
    m, off = [], 0
    for k in range(g.d):
        sz = int(np.prod(g.m_shape(k)))
        m.append(vec[off:off + sz].reshape(g.m_shape(k)))
        off += sz
    f = vec[off:off + int(np.prod(g.f_shape))].reshape(g.f_shape)
    return m, f


def pack_dual(g, bm, bf):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in bm] + [np.asarray(bf, np.float64).ravel()])


def unpack_dual(g, vec):
    n = g.ncells
    parts = [vec[i * n:(i + 1) * n].reshape(g.cell_shape) for i in range(g.d + 1)]
    return parts[:-1], parts[-1]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32(a):
    return np.ascontiguousarray(np.asarray(a, np.float32))


def random_pair(g, seed, floor=0.2):
    rng = np.random.default_rng(seed)
    f0 = rng.random(g.space_shape) + floor
    f1 = rng.random(g.space_shape) + floor
    f0 = f0.astype(np.float32).astype(np.float64)
    f1 = (f1 * (f0.sum() / f1.sum())).astype(np.float32).astype(np.float64)
    return f0, f1


EPS32 = 2.0 ** -24


def smooth_field(shape, rng, nterms=12, kmax=4):
    """Random smooth field: a sum of separable low-frequency cosines."""
    out = np.zeros(shape)
    for _ in range(nterms):
        term = np.full(shape, rng.standard_normal())
        for ax, s in enumerate(shape):
            k = int(rng.integers(0, kmax + 1))
            ph = rng.uniform(0, 2 * np.pi)
            v = np.cos(np.pi * k * (np.arange(s) + 0.5) / s + ph)
            sh = [1] * len(shape)
            sh[ax] = s
            term = term * v.reshape(sh)
        out += term
    return out


def correction_tolerance(g, phi, x_vec, c=10.0):
    """Relative error bound of x = a - A^T phi in FP32 for a given input.

    The inverse transforms leave a rounding error of relative size ~c eps32 in
    phi, spread over all modes; A^T amplifies it by up to sqrt(lambda_max), so
    the error of x relative to ||x|| is about c eps32 sqrt(lambda_max) ||phi|| / ||x||.
    """
    lam_max = float(o.eigenvalues(g).max())
    kappa = np.sqrt(lam_max) * np.linalg.norm(phi) / max(np.linalg.norm(x_vec), 1e-300)
    return 1e-5 + c * EPS32 * kappa
