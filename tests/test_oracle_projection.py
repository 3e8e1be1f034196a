"""Pins of the oracle's projection onto C_d (section 3, step 1) against dense
linear algebra: the eigenvalues of A A^T from numpy.linalg.eigvalsh, the
pseudo-inverse from numpy.linalg.pinv and the minimum-norm correction from
numpy.linalg.lstsq, on grids small enough for dense matrices."""
import numpy as np
import pytest

import oracle as o
from test_oracle_operators import GRIDS, dense_ops, fb_dense


def dense_A(g):
    SM, SF, DM, DF = dense_ops(g)
    return np.hstack(DM + [DF])


def flat_x(g, m, f):
    return np.concatenate([a.ravel() for a in m] + [f.ravel()])


def unflat_x(g, x):
    m, off = [], 0
    for k in range(g.d):
        sz = int(np.prod(g.m_shape(k)))
        m.append(x[off:off + sz].reshape(g.m_shape(k)))
        off += sz
    return m, x[off:].reshape(g.f_shape)


IDS = lambda g: "x".join(map(str, g.n)) + "_" + "".join(b[0] for b in g.bc) + "_P%d" % g.P


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_eigenvalues_match_dense(g):
    Ad = dense_A(g)
    ev = np.sort(np.linalg.eigvalsh(Ad @ Ad.T))
    lam = np.sort(o.eigenvalues(g).ravel())
    np.testing.assert_allclose(lam, ev, rtol=1e-10, atol=1e-9)
    assert abs(lam[0]) < 1e-9 and lam[1] > 1e-3   # one zero mode


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_projection_matches_pinv_and_lstsq(g):
    rng = np.random.default_rng(5)
    Ad = dense_A(g)
    f0 = rng.random(g.space_shape) + 0.1
    f1 = rng.random(g.space_shape) + 0.1
    f1 *= f0.sum() / f1.sum()
    _, fbm = fb_dense(g, f0, f1)
    am = [rng.standard_normal(g.m_shape(k)) for k in range(g.d)]
    af = rng.standard_normal(g.f_shape)
    a = flat_x(g, am, af)
    x_pinv = a - Ad.T @ (np.linalg.pinv(Ad @ Ad.T, rcond=1e-10, hermitian=True) @ (Ad @ a - fbm))
    x_lsq = a + np.linalg.lstsq(Ad, fbm - Ad @ a, rcond=None)[0]
    m, f, phi = o.project(g, am, af, f0, f1)
    x = flat_x(g, m, f)
    np.testing.assert_allclose(x, x_pinv, rtol=0, atol=1e-10 * max(1, np.abs(x_pinv).max()))
    np.testing.assert_allclose(x, x_lsq, rtol=0, atol=1e-10 * max(1, np.abs(x_pinv).max()))
    # the result lies in C_d and the projection is idempotent
    np.testing.assert_allclose(Ad @ x, fbm, atol=1e-9 * max(1, np.abs(fbm).max()))
    m2, f2, _ = o.project(g, m, f, f0, f1)
    np.testing.assert_allclose(flat_x(g, m2, f2), x, atol=1e-10 * max(1, np.abs(x).max()))


@pytest.mark.parametrize("g", GRIDS, ids=IDS)
def test_poisson_pinv_matches_dense(g):
    rng = np.random.default_rng(7)
    Ad = dense_A(g)
    r = rng.standard_normal(g.cell_shape)
    phi = o.poisson_pinv(g, r)
    ref = np.linalg.pinv(Ad @ Ad.T, rcond=1e-10, hermitian=True) @ r.ravel()
    np.testing.assert_allclose(phi.ravel(), ref, atol=1e-10 * max(1, np.abs(ref).max()))


def test_projection_preserves_mass_per_time():
    """Summing A x = f_b^- over space gives p (sum f_k - sum f_{k-1}) = 0."""
    g = o.rgb_grid(6, 5, 7)
    rng = np.random.default_rng(9)
    f0 = rng.random(g.space_shape)
    f1 = rng.random(g.space_shape)
    f1 *= f0.sum() / f1.sum()
    am = [rng.standard_normal(g.m_shape(k)) for k in range(g.d)]
    af = rng.standard_normal(g.f_shape)
    m, f, _ = o.project(g, am, af, f0, f1)
    sums = f.reshape(g.P - 1, -1).sum(axis=1)
    np.testing.assert_allclose(sums, f0.sum(), rtol=1e-12)
