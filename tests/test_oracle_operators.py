"""Pins of the oracle's stencil operators against dense matrices built
literally from the paper's printed definitions (section 2: S_n, S_{n,per},
S_p, D_{n,per}, D_p, Kronecker forms of S_M, S_F, D_M, D_F and f_b^+-).

Readings of garbled entries: the last rows of S_{n,per} and D_{n,per} are read
as the cyclic bidiagonal continuation of the other rows; D_n and S_n (not
printed) follow the pattern of D_p and S_p with n in place of p.
"""
import numpy as np
import pytest

import oracle as o

# ---- dense matrices, written from the paper's matrices ---------------------


def S_p_dense(p):
    """S_p = 1/2 [[1 1 . .], [. 1 1 .], ...] in R^{p-1, p}."""
    S = np.zeros((p - 1, p))
    for l in range(p - 1):
        S[l, l] = S[l, l + 1] = 0.5
    return S


def D_p_dense(p, scale=None):
    """D_p = p [[-1 1 . .], [. -1 1 .], ...] in R^{p-1, p}."""
    s = p if scale is None else scale
    D = np.zeros((p - 1, p))
    for l in range(p - 1):
        D[l, l] = -s
        D[l, l + 1] = s
    return D


def S_nper_dense(n):
    """S_{n,per} = 1/2 (first row (1, 0, ..., 0, 1), row i: ones at i-1, i)."""
    S = np.zeros((n, n))
    S[0, 0] += 0.5
    S[0, n - 1] += 0.5
    for i in range(1, n):
        S[i, i - 1] += 0.5
        S[i, i] += 0.5
    return S


def D_nper_dense(n, scale=None):
    """D_{n,per} = n (first row (-1, 0, ..., 0, 1), row i: 1 at i-1, -1 at i)."""
    s = n if scale is None else scale
    D = np.zeros((n, n))
    D[0, 0] += -s
    D[0, n - 1] += s
    for i in range(1, n):
        D[i, i - 1] += s
        D[i, i] += -s
    return D


def read_golden(name):
    """Matrices of a text fixture under tests/golden: a header line 'name rows cols', then the rows."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    lines = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    out, i = {}, 0
    while i < len(lines):
        key, r, c = lines[i][0], int(lines[i][1]), int(lines[i][2])
        out[key] = np.array([[float(v) for v in lines[i + 1 + j]] for j in range(r)]).reshape(r, c)
        i += 1 + r
    return out


def test_dense_builders_match_the_printed_matrices():
    """The builders above against the section 2 matrices written out by hand at p = 3, n = 4
    (tests/golden/operators_p3_n4.txt), and Remark 2's colour eigenvalues."""
    gold = read_golden("operators_p3_n4.txt")
    np.testing.assert_array_equal(S_p_dense(3), gold["S_p"])
    np.testing.assert_array_equal(D_p_dense(3), gold["D_p"])
    np.testing.assert_array_equal(S_nper_dense(4), gold["S_nper"])
    np.testing.assert_array_equal(D_nper_dense(4), gold["D_nper"])
    Dc = D_nper_dense(3, scale=1.0)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Dc.T @ Dc)), gold["eig_colour_laplacian_3"][0], atol=1e-12)


def space_factor(g, k, M):
    """I (x) ... (x) M (x) ... (x) I acting on spatial axis k (x fastest)."""
    out = np.ones((1, 1))
    for kk in reversed(range(g.d)):          # slowest spatial axis first
        out = np.kron(out, M if kk == k else np.eye(g.n[kk]))
    return out


def dense_ops(g):
    """Dense S_M (list per axis), S_F, D_M (list per axis), D_F."""
    P = g.P
    SM, DM = [], []
    for k in range(g.d):
        n = g.n[k]
        if g.bc[k] == o.NEUMANN:
            Sk = S_p_dense(n).T                # S_n^T
            Dk = -D_p_dense(n, g.scale[k]).T   # -D_n^T
        else:
            Sk = S_nper_dense(n).T
            Dk = D_nper_dense(n, g.scale[k]).T
        SM.append(np.kron(np.eye(P), space_factor(g, k, Sk)))
        DM.append(np.kron(np.eye(P), space_factor(g, k, Dk)))
    In = np.eye(g.npix)
    SF = np.kron(S_p_dense(P).T, In)
    DF = np.kron(-D_p_dense(P).T, In)
    return SM, SF, DM, DF


def fb_dense(g, f0, f1):
    P, n = g.P, g.npix
    plus = 0.5 * np.concatenate([f0.ravel(), np.zeros(n * (P - 2)), f1.ravel()])
    minus = P * np.concatenate([f0.ravel(), np.zeros(n * (P - 2)), -f1.ravel()])
    return plus, minus


GRIDS = [
    o.Grid((5,), (o.NEUMANN,), 4),
    o.Grid((6,), (o.PERIODIC,), 3),
    o.Grid((5,), (o.PERIODIC,), 5),
    o.rgb_grid(3, 4, 3),
    o.Grid((4, 3, 3), (o.NEUMANN, o.NEUMANN, o.NEUMANN), 3),
    o.Grid((4, 3), (o.PERIODIC, o.NEUMANN), 4, scale=(2.5, 7.0)),
]


def _rand_state(g, rng):
    m = [rng.standard_normal(g.m_shape(k)) for k in range(g.d)]
    f = rng.standard_normal(g.f_shape)
    return m, f


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: "x".join(map(str, g.n)) + "_" + "".join(b[0] for b in g.bc) + "_P%d" % g.P)
def test_operators_match_dense(g):
    rng = np.random.default_rng(1)
    SM, SF, DM, DF = dense_ops(g)
    m, f = _rand_state(g, rng)
    u = o.S_M(g, m)
    for k in range(g.d):
        np.testing.assert_allclose(u[k].ravel(), SM[k] @ m[k].ravel(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(o.S_F(g, f).ravel(), SF @ f.ravel(), rtol=0, atol=1e-14)
    div = sum(DM[k] @ m[k].ravel() for k in range(g.d)) + DF @ f.ravel()
    np.testing.assert_allclose(o.A(g, m, f).ravel(), div, rtol=0, atol=1e-12)
    # adjoints
    w = [rng.standard_normal(g.cell_shape) for _ in range(g.d)]
    wt = o.S_M_T(g, w)
    for k in range(g.d):
        np.testing.assert_allclose(wt[k].ravel(), SM[k].T @ w[k].ravel(), rtol=0, atol=1e-14)
    vf = rng.standard_normal(g.cell_shape)
    np.testing.assert_allclose(o.S_F_T(g, vf).ravel(), SF.T @ vf.ravel(), rtol=0, atol=1e-14)
    phi = rng.standard_normal(g.cell_shape)
    mt, ft = o.A_T(g, phi)
    for k in range(g.d):
        np.testing.assert_allclose(mt[k].ravel(), DM[k].T @ phi.ravel(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(ft.ravel(), DF.T @ phi.ravel(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("g", GRIDS[:4])
def test_boundary_vectors(g):
    rng = np.random.default_rng(2)
    f0 = rng.random(g.space_shape)
    f1 = rng.random(g.space_shape)
    plus, minus = fb_dense(g, f0, f1)
    np.testing.assert_allclose(o.f_b_plus(g, f0, f1).ravel(), plus, atol=1e-15)
    np.testing.assert_allclose(o.f_b_minus(g, f0, f1).ravel(), minus, atol=1e-13)


def test_continuity_is_forward_difference_in_time():
    """A x = f_b^- reads p (f_k - f_{k-1}) + div m = 0 with f_0 = f0, f_p = f1."""
    g = o.Grid((4,), (o.NEUMANN,), 3)
    rng = np.random.default_rng(3)
    f0, f1 = rng.random(4), rng.random(4)
    m, f = _rand_state(g, rng)
    r = o.A(g, m, f) - o.f_b_minus(g, f0, f1)
    F = np.concatenate([f0[None], f, f1[None]])
    mfull = np.concatenate([np.zeros((3, 1)), m[0], np.zeros((3, 1))], axis=1)
    expect = 3 * (F[1:] - F[:-1]) + 4 * (mfull[:, 1:] - mfull[:, :-1])
    np.testing.assert_allclose(r, expect, atol=1e-13)


def test_periodic_even_null_space_of_S_M():
    """Theorem 1 proof: for periodic BC and even n, N(S_M) = {w (x) (1,-1,...)}."""
    for n, expect_dim in [(6, 1), (5, 0)]:
        S = S_nper_dense(n).T
        sv = np.linalg.svd(S, compute_uv=False)
        assert int(np.sum(sv < 1e-12)) == expect_dim
    g = o.Grid((6,), (o.PERIODIC,), 3)
    w = np.array([0.3, -1.0, 2.0])
    alt = np.array([1, -1, 1, -1, 1, -1], dtype=float)
    m = [w[:, None] * alt[None, :]]
    u = o.S_M(g, m)
    assert np.abs(u[0]).max() < 1e-15
