"""Pins of the oracle's full iteration (Algorithm 1) against facts the paper
and the mathematics fix: mass conservation per time slice (from C_d), the
zero-energy cases f0 = f1 and Remark 1, equivariance under a cyclic colour
shift and under time reversal, translation of a blob, the 1D quantile
closed form of optimal transport on the line (section 1), and the vanishing of
the primal-dual gap at the saddle point."""
import numpy as np

import oracle as o

SIG = 0.3


def _pair(g, seed, floor=0.2):
    rng = np.random.default_rng(seed)
    f0 = rng.random(g.space_shape) + floor
    f1 = rng.random(g.space_shape) + floor
    f1 *= f0.sum() / f1.sum()
    return f0, f1


def test_mass_per_time_slice_every_iteration():
    g = o.rgb_grid(7, 5, 6)
    f0, f1 = _pair(g, 0)
    g0, g1, _ = o.normalise_pair(g, f0, f1)
    st = o.State.zeros(g)
    for _ in range(25):
        st, info = o.pdhg_step(g, st, g0, g1, SIG, 0.99 / SIG)
        sums = st.f.reshape(g.P - 1, -1).sum(axis=1)
        np.testing.assert_allclose(sums, g0.sum(), rtol=1e-12)
        assert info.continuity < 1e-13


def test_equal_endpoints_give_zero_energy():
    g = o.rgb_grid(6, 6, 5)
    f0, _ = _pair(g, 1)
    st, infos, _ = o.solve(g, f0, f0.copy(), 1600, SIG, 0.99 / SIG)
    g0, _, _ = o.normalise_pair(g, f0, f0)
    assert infos[-1].energy < 1e-12
    for k in range(g.P - 1):
        np.testing.assert_allclose(st.f[k], g0, rtol=0, atol=1e-4)
    assert max(np.abs(m).max() for m in st.m) < 1e-4


def test_primal_dual_gap_vanishes_at_convergence():
    """At a saddle point the energy of the prox output equals the dual value: J is 1-homogeneous, so
    J(y) = <p, y> for p = sigma b in its subdifferential (step 2), y = K x + (0, f_b^+) (step 3 at a
    fixed point), and K^T p lies in the range of A^T (optimality over C_d), where <K^T p, x> = <K^T p, x0>.
    Solved to a splitting residual of 1e-11 the gap is below 1e-8 of the energy; early iterates have a
    gap of order one or more."""
    g = o.rgb_grid(6, 5, 4)
    f0, f1 = _pair(g, 3, floor=0.3)
    st, infos, _ = o.solve(g, f0, f1, 6000, SIG, 0.99 / SIG, with_dual=True, tol=1e-11, check_every=10)
    last = infos[-1]
    assert last.residual <= 1e-11
    assert abs(last.energy - last.dual) <= 1e-8 * last.energy
    assert abs(infos[0].energy - infos[0].dual) > 0.5 * infos[0].energy


def test_primal_dual_gap_with_equal_endpoints():
    """f0 = f1: the optimal energy is zero, and so is the dual value of the converged dual."""
    g = o.rgb_grid(6, 6, 5)
    f0, _ = _pair(g, 1)
    _, infos, _ = o.solve(g, f0, f0.copy(), 1600, SIG, 0.99 / SIG, with_dual=True)
    assert infos[-1].energy < 1e-12 and abs(infos[-1].dual) < 1e-10


def test_min_norm_path_is_the_nearest_feasible_path():
    """x0 = Pi_{C_d}(0) meets the continuity constraint and is orthogonal to ker A (so no feasible path is
    shorter): every other feasible path x0 + w (w in ker A) is longer, with <x0, w> = 0."""
    g = o.rgb_grid(5, 4, 4)
    f0, f1 = _pair(g, 8)
    g0, g1, _ = o.normalise_pair(g, f0, f1)
    m0, fz = o.min_norm_path(g, g0, g1)
    fbm = o.f_b_minus(g, g0, g1)
    assert np.abs(o.A(g, m0, fz) - fbm).max() < 1e-12
    n0 = sum(float(np.sum(a * a)) for a in m0) + float(np.sum(fz * fz))
    rng = np.random.default_rng(9)
    for _ in range(3):
        zm = [rng.standard_normal(g.m_shape(k)) for k in range(g.d)]
        zf = rng.standard_normal(g.f_shape)
        pm, pf, _ = o.project(g, [a + b for a, b in zip(m0, zm)], fz + zf, g0, g1)   # another feasible path
        n1 = sum(float(np.sum(a * a)) for a in pm) + float(np.sum(pf * pf))
        inner = sum(float(np.sum(a * (b - a))) for a, b in zip(m0, pm)) + float(np.sum(fz * (pf - fz)))
        assert n1 > n0 and abs(inner) < 1e-9 * n0


def test_remark1_nonunique_zero_energy():
    """Periodic even n, f1 = f0 + gamma (1,-1,...): a zero-energy minimiser exists."""
    g = o.Grid((6,), (o.PERIODIC,), 4)
    f0 = np.array([1.0, 1.2, 0.9, 1.1, 1.3, 0.8])
    alt = np.array([1, -1, 1, -1, 1, -1], dtype=float)
    f1 = f0 + 0.5 * alt
    st, infos, _ = o.solve(g, f0, f1, 3000, SIG, 0.99 / SIG, normalise=False)
    assert infos[-1].energy < 1e-6
    # and the transport indeed uses the null space: u = S_M m ~ 0 while m != 0
    u = o.S_M(g, st.m)[0]
    assert np.abs(u).max() < 1e-2 * np.abs(st.m[0]).max()


def test_colour_shift_equivariance():
    """Periodic colour: rolling the channels of f0, f1 rolls every iterate."""
    g = o.rgb_grid(5, 4, 4)
    f0, f1 = _pair(g, 2)
    r0, r1 = np.roll(f0, 1, axis=0), np.roll(f1, 1, axis=0)
    sa = o.State.zeros(g)
    sb = o.State.zeros(g)
    g0, g1, _ = o.normalise_pair(g, f0, f1)
    h0, h1, _ = o.normalise_pair(g, r0, r1)
    cax = g.ax(2)
    for _ in range(15):
        sa, _ = o.pdhg_step(g, sa, g0, g1, SIG, 0.99 / SIG)
        sb, _ = o.pdhg_step(g, sb, h0, h1, SIG, 0.99 / SIG)
        np.testing.assert_allclose(sb.f, np.roll(sa.f, 1, axis=cax), atol=1e-12)
        for k in range(3):
            np.testing.assert_allclose(sb.m[k], np.roll(sa.m[k], 1, axis=cax), atol=1e-12)


def test_neumann_colour_is_not_shift_equivariant():
    """Section 1 / Fig. 1: with Neumann colour the result depends on channel order."""
    g = o.Grid((5, 4, 3), (o.NEUMANN, o.NEUMANN, o.NEUMANN), 4)
    f0, f1 = _pair(g, 2)
    g0, g1, _ = o.normalise_pair(g, f0, f1)
    h0, h1, _ = o.normalise_pair(g, np.roll(f0, 1, axis=0), np.roll(f1, 1, axis=0))
    sa, _, _ = o.solve(g, g0, g1, 30, SIG, 0.99 / SIG, normalise=False)
    sb, _, _ = o.solve(g, h0, h1, 30, SIG, 0.99 / SIG, normalise=False)
    assert np.abs(sb.f - np.roll(sa.f, 1, axis=1)).max() > 1e-3


def test_time_reversal_equivariance():
    """Swapping f0 and f1 reverses f in time and negates and reverses m."""
    g = o.rgb_grid(5, 4, 5)
    f0, f1 = _pair(g, 3)
    sa, _, _ = o.solve(g, f0, f1, 12, SIG, 0.99 / SIG)
    sb, _, _ = o.solve(g, f1, f0, 12, SIG, 0.99 / SIG)
    np.testing.assert_allclose(sb.f, sa.f[::-1], atol=1e-11)
    for k in range(3):
        np.testing.assert_allclose(sb.m[k], -sa.m[k][::-1], atol=1e-11)


def _bump(x, c, w):
    return np.exp(-0.5 * ((x - c) / w) ** 2)


def test_quantile_closed_form_1d_neumann():
    """OT on the line: F_t^{-1} = (1-t) F_0^{-1} + t F_1^{-1}, E = W2^2 / 2."""
    n, P = 96, 16
    g = o.Grid((n,), (o.NEUMANN,), P)
    x = (np.arange(n) + 0.5) / n
    f0 = _bump(x, 0.3, 0.06) + 0.6 * _bump(x, 0.45, 0.04) + 0.05
    f1 = _bump(x, 0.65, 0.08) + 0.05
    f0 *= n / f0.sum()
    f1 *= n / f1.sum()
    st, infos, _ = o.solve(g, f0, f1, 2500, SIG, 0.99 / SIG, normalise=False)
    # closed form on a fine quantile grid, from the piecewise-constant densities
    q = (np.arange(4000) + 0.5) / 4000

    def qf(dens):
        cdf = np.concatenate([[0.0], np.cumsum(dens) / dens.sum()])
        edges = np.arange(n + 1) / n
        return np.interp(q, cdf, edges)

    Q0, Q1 = qf(f0), qf(f1)
    W2sq = np.mean((Q1 - Q0) ** 2)
    E = infos[-1].energy
    assert abs(E - 0.5 * W2sq) < 0.03 * 0.5 * W2sq
    # the dual value of the final dual iterate approaches the same optimal value
    x0 = o.min_norm_path(g, f0, f1)
    D = o.dual_value(g, st.bm, st.bf, x0, f0, f1, SIG)
    assert abs(D - 0.5 * W2sq) < 0.03 * 0.5 * W2sq
    # CDF of the discrete f at t = k/P against the closed-form CDF
    for k in [P // 4, P // 2, 3 * P // 4]:
        t = k / P
        Qt = (1 - t) * Q0 + t * Q1
        edges = np.arange(n + 1) / n
        cdf_closed = np.interp(edges, np.concatenate([[0], Qt, [1]]), np.concatenate([[0], q, [1]]))
        cdf_disc = np.concatenate([[0.0], np.cumsum(st.f[k - 1])]) / st.f[k - 1].sum()
        assert np.abs(cdf_disc - cdf_closed).max() < 0.03


def test_translation_energy_and_centroid():
    """A blob shifted by s cells (2D grey, Neumann): E ~ |s/n|^2 / 2, centroid linear in t."""
    n, P, s = 32, 8, 6
    g = o.Grid((n, n), (o.NEUMANN, o.NEUMANN), P)
    yy, xx = np.meshgrid((np.arange(n) + 0.5), (np.arange(n) + 0.5), indexing="ij")
    f0 = np.exp(-((xx - 12) ** 2 + (yy - 16) ** 2) / (2 * 3.0 ** 2)) + 1e-3
    f1 = np.exp(-((xx - 12 - s) ** 2 + (yy - 16) ** 2) / (2 * 3.0 ** 2)) + 1e-3
    f1 *= f0.sum() / f1.sum()
    st, infos, _ = o.solve(g, f0, f1, 1500, SIG, 0.99 / SIG)
    E = infos[-1].energy
    expect = 0.5 * (s / n) ** 2
    assert abs(E - expect) < 0.05 * expect
    g0, _, _ = o.normalise_pair(g, f0, f1)
    cx0 = (g0 * xx).sum() / g0.sum()
    for k in range(1, P):
        cx = (st.f[k - 1] * xx).sum() / st.f[k - 1].sum()
        assert abs(cx - (cx0 + s * k / P)) < 0.1


def test_warm_state_dual_is_the_converged_dual():
    """At a fixed point of Algorithm 1 the dual equals grad J(K x + (0, f_b^+)) / sigma
    (optimality of step 2 with y = K x + (0, f_b^+)); a warm state built from the
    converged path therefore reproduces the converged dual and is itself a fixed point."""
    g = o.rgb_grid(6, 5, 4)
    f0, f1 = _pair(g, 11, floor=0.5)
    g0, g1, _ = o.normalise_pair(g, f0, f1)
    st, infos, _ = o.solve(g, f0, f1, 3000, SIG, 0.99 / SIG)
    assert infos[-1].residual < 1e-9
    w = o.warm_state(g, st.m, st.f, g0, g1, SIG)
    ref = st.bm + [st.bf]
    got = w.bm + [w.bf]
    for a, b in zip(got, ref):
        np.testing.assert_allclose(a, b, atol=1e-7 * max(1.0, np.abs(b).max()))
    _, info = o.pdhg_step(g, w, g0, g1, SIG, 0.99 / SIG)
    assert info.residual < 1e-7
    # without the dual the first step moves b by O(1)
    _, info0 = o.pdhg_step(g, o.warm_state(g, st.m, st.f, g0, g1, SIG, dual=False), g0, g1, SIG, 0.99 / SIG)
    assert info0.residual > 1e-3
    z = o.warm_state(g, st.m, st.f, g0, g1, SIG, dual=False)
    assert all(not a.any() for a in z.bm + [z.bf] + z.bbm + [z.bbf])


def _fig1_pair(n):
    """A Gaussian that is red at t = 0 and blue at t = 1 (section 1, Fig. 1), on a small floor."""
    yy, xx = np.mgrid[0:n, 0:n] + 0.5
    gauss = np.exp(-((xx - n / 2) ** 2 + (yy - n / 2) ** 2) / (2 * 2.0 ** 2))

    def img(ch):
        f = np.full((3, n, n), 1e-3)
        f[ch] += gauss
        return f / f.sum()
    return img(0), img(2)


def test_fig1_red_to_blue_colour_boundary():
    """Fig. 1: with periodic colour, red reaches blue directly (red and blue are neighbours on the
    colour circle), so little mass passes through green at t = 1/2; with Neumann colour the path
    from red to blue runs through green, which then holds most of the mass."""
    n, P = 12, 8
    f0, f1 = _fig1_pair(n)
    frac = {}
    for bc in ("periodic", "neumann"):
        g = o.Grid((n, n, 3), ("neumann", "neumann", bc), P)
        st, _, sc = o.solve(g, f0, f1, 800, SIG, 0.99 / SIG)
        mid = st.f[P // 2 - 1] * sc                      # f at time 1/2
        frac[bc] = mid.sum(axis=(1, 2)) / mid.sum()
    assert frac["periodic"][1] < 0.15 and abs(frac["periodic"][0] - frac["periodic"][2]) < 1e-6
    assert frac["neumann"][1] > 0.5
