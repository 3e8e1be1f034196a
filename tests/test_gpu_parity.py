"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

The prox and the Poisson solve phi = (A A^T)^+ r agree to 1e-5 relative L2.
The projection x = a - A^T phi and whole iterations agree to the FP32 bound of
the correction A^T phi (tests/_helpers.correction_tolerance: 1e-5 plus ten
float32 epsilons times the amplification sqrt(lambda_max) ||phi|| / ||x||), and
a full solve at a fixed iteration count to 1e-3 relative L2 of f.
Grids cover several tiles and ragged tails: power-of-two FFT lengths, dense
lengths, odd P, grey and 1D Neumann problems, Neumann colour, hue histograms
of even and odd length, and the full 256 x 256 x 3 x 32 benchmark size."""
import numpy as np
import pytest

import oracle as o
from _helpers import (correction_tolerance, f32, oracle_grid, pack_dual, pack_path, random_pair, rel, smooth_field,
                      unpack_dual, unpack_path)

pytestmark = pytest.mark.gpu

SIG = 0.3
TAU = 0.99 / 0.3


@pytest.fixture(scope="module")
def ot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_04840_gb300 import _build
    _build.build()
    import paper_1501_04840_gb300 as p
    p.load_library()
    return p


def make_plan(ot, n, bc, P, batch=1, precision=0):
    g = ot.grid(n, bc, P, sigma=SIG, tau=TAU, precision=precision)
    return ot.Plan(g, batch=batch), oracle_grid(n, bc, P)


RGB = ("neumann", "neumann", "periodic")
GRIDS = [
    ((32, 32, 3), RGB, 16),
    ((64, 64, 3), RGB, 16),
    ((48, 40, 3), RGB, 12),
    ((128, 96, 3), RGB, 17),
    ((64, 128, 3), RGB, 7),
    ((64, 48), ("neumann", "neumann"), 8),
    ((96,), ("neumann",), 16),
    ((32, 24, 3), ("neumann", "neumann", "neumann"), 6),
    ((360,), ("periodic",), 64),
    ((101,), ("periodic",), 20),
    ((2, 2, 3), RGB, 2),
    ((24, 20, 3), ("periodic", "periodic", "periodic"), 8),
    ((32, 16, 3), ("periodic", "neumann", "periodic"), 6),
    ((16, 24), ("neumann", "periodic"), 5),
    ((33, 7), ("periodic", "periodic"), 4),
    ((64, 128, 3), ("periodic", "periodic", "periodic"), 8),
    ((256, 64, 3), ("periodic", "neumann", "periodic"), 4),
    ((128, 64), ("neumann", "periodic"), 6),
    ((192, 96, 3), RGB, 16),
    ((96, 192, 3), ("periodic", "periodic", "periodic"), 8),
    ((192, 64), ("periodic", "neumann"), 6),
    ((256, 256, 3), RGB, 32),
]
IDS = ["x".join(map(str, n)) + "_" + "".join(b[0] for b in bc) + "_P%d" % P for n, bc, P in GRIDS]


def test_prox_matches_oracle(ot):
    rng = np.random.default_rng(0)
    n = 200_000
    am = (rng.standard_normal((3, n)) * rng.choice([0.01, 1.0, 30.0], size=n)).astype(np.float32)
    af = (rng.standard_normal(n) * rng.choice([0.01, 1.0, 30.0], size=n)).astype(np.float32)
    u, v = ot.prox(am, af, SIG)
    uo, vo = o.prox_J([am[k].astype(np.float64) for k in range(3)], af.astype(np.float64), SIG)
    assert rel(v, vo) <= 1e-5
    assert rel(u, np.stack(uo)) <= 1e-5
    # the zero branch is exact
    zero = (af.astype(np.float64) + 0.5 * SIG * (am.astype(np.float64) ** 2).sum(0)) <= 0
    assert np.all(v[zero] == 0) and np.all(u[:, zero] == 0)


def test_prox_cardano_against_newton_and_oracle(ot):
    """The closed-form prox (Cardano) against the FP64 oracle on the same mix of scales as the Newton
    test: relative L2 within 1e-5 too, and per-cell errors reported for both methods.  The closed form
    loses relative accuracy where the root sits just above the edge of the feasible set (small d with
    c < 0: three real roots, arccos near its end), which Newton's scale-aware stop does not."""
    rng = np.random.default_rng(1)
    n = 200_000
    am = (rng.standard_normal((3, n)) * rng.choice([0.01, 1.0, 30.0], size=n)).astype(np.float32)
    af = (rng.standard_normal(n) * rng.choice([0.01, 1.0, 30.0], size=n)).astype(np.float32)
    uo, vo = o.prox_J([am[k].astype(np.float64) for k in range(3)], af.astype(np.float64), SIG)
    errs = {}
    for method in ("newton", "cardano"):
        u, v = ot.prox(am, af, SIG, method=method)
        errs[method] = (rel(v, vo), rel(u, np.stack(uo)))
        scale = np.abs(vo) + np.abs(af) + 1e-30
        errs[method] += (float(np.max(np.abs(v - vo) / scale)),)
    print("prox errors (rel L2 v, rel L2 u, max |dv| / (|v| + |a_f|)):", errs)
    assert errs["cardano"][0] <= 1e-5 and errs["cardano"][1] <= 1e-5
    assert errs["newton"][0] <= 1e-5 and errs["newton"][1] <= 1e-5


@pytest.mark.parametrize("n,bc,P", GRIDS, ids=IDS)
def test_projection_matches_oracle(ot, n, bc, P):
    """Smooth operands: phi to 1e-5; x to the FP32 bound of the A^T phi correction."""
    plan, g = make_plan(ot, n, bc, P)
    rng = np.random.default_rng(1)
    f0, f1 = random_pair(g, 2)
    am = [smooth_field(g.m_shape(k), rng).astype(np.float32).astype(np.float64) for k in range(g.d)]
    af = smooth_field(g.f_shape, rng).astype(np.float32).astype(np.float64)
    x, phi = plan.project(f32(f0), f32(f1), f32(pack_path(g, am, af)), with_phi=True)
    m, f, phio = o.project(g, am, af, f0, f1)
    xo = pack_path(g, m, f)
    assert rel(phi, phio.ravel()) <= 1e-5
    assert rel(x, xo) <= correction_tolerance(g, phio, xo)


@pytest.mark.parametrize("n,bc,P", GRIDS, ids=IDS)
def test_projection_white_noise(ot, n, bc, P):
    """White-noise operands: phi to 1e-5; x to the FP32 bound of the A^T phi correction."""
    plan, g = make_plan(ot, n, bc, P)
    rng = np.random.default_rng(11)
    f0, f1 = random_pair(g, 2)
    am = [rng.standard_normal(g.m_shape(k)).astype(np.float32).astype(np.float64) for k in range(g.d)]
    af = rng.standard_normal(g.f_shape).astype(np.float32).astype(np.float64)
    x, phi = plan.project(f32(f0), f32(f1), f32(pack_path(g, am, af)), with_phi=True)
    m, f, phio = o.project(g, am, af, f0, f1)
    xo = pack_path(g, m, f)
    assert rel(phi, phio.ravel()) <= 1e-5
    assert rel(x, xo) <= correction_tolerance(g, phio, xo)


def _random_state(g, seed, smooth=False):
    rng = np.random.default_rng(seed)
    gen = (lambda shape: smooth_field(shape, rng)) if smooth else (lambda shape: rng.standard_normal(shape))
    st = o.State.zeros(g)
    st.m = [gen(g.m_shape(k)) for k in range(g.d)]
    st.f = np.abs(gen(g.f_shape)) + 0.1
    st.bm = [0.3 * gen(g.cell_shape) for _ in range(g.d)]
    st.bf = 0.3 * gen(g.cell_shape)
    st.bbm = [0.3 * gen(g.cell_shape) for _ in range(g.d)]
    st.bbf = 0.3 * gen(g.cell_shape)
    # round through float32 so both sides start from identical values
    st.m = [a.astype(np.float32).astype(np.float64) for a in st.m]
    st.f = st.f.astype(np.float32).astype(np.float64)
    for name in ("bm", "bbm"):
        setattr(st, name, [a.astype(np.float32).astype(np.float64) for a in getattr(st, name)])
    st.bf = st.bf.astype(np.float32).astype(np.float64)
    st.bbf = st.bbf.astype(np.float32).astype(np.float64)
    return st


def _step_tolerance(g, st, f0, f1):
    """The projection inside the step bounds its FP32 error (see correction_tolerance)."""
    km, kf = o.K_T(g, st.bbm, st.bbf)
    am = [st.m[k] - TAU * SIG * km[k] for k in range(g.d)]
    af = st.f - TAU * SIG * kf
    mm, ff, phio = o.project(g, am, af, f0, f1)
    return correction_tolerance(g, phio, pack_path(g, mm, ff))


def _one_iteration(ot, n, bc, P, smooth, seed=4):
    plan, g = make_plan(ot, n, bc, P)
    f0, f1 = random_pair(g, 3)
    st = _random_state(g, seed, smooth)
    plan.state_set(f32(f0), f32(f1), f32(pack_path(g, st.m, st.f)), f32(pack_dual(g, st.bm, st.bf)),
                   f32(pack_dual(g, st.bbm, st.bbf)))
    plan.iterate(1)
    x, b, bb = plan.state_get()
    new, _ = o.pdhg_step(g, st, f0, f1, SIG, TAU)
    tol = _step_tolerance(g, st, f0, f1)
    m, f = unpack_path(g, x.astype(np.float64))
    assert rel(f, new.f) <= tol
    for k in range(g.d):
        assert rel(m[k], new.m[k]) <= tol
    bm, bf = unpack_dual(g, b.astype(np.float64))
    bbm, bbf = unpack_dual(g, bb.astype(np.float64))
    assert rel(bf, new.bf) <= tol and rel(bbf, new.bbf) <= tol
    for k in range(g.d):
        assert rel(bm[k], new.bm[k]) <= tol and rel(bbm[k], new.bbm[k]) <= tol


@pytest.mark.parametrize("n,bc,P", GRIDS, ids=IDS)
def test_one_iteration_matches_oracle(ot, n, bc, P):
    _one_iteration(ot, n, bc, P, smooth=True)


@pytest.mark.parametrize("n,bc,P", GRIDS, ids=IDS)
def test_one_iteration_white_noise_state(ot, n, bc, P):
    _one_iteration(ot, n, bc, P, smooth=False)


def test_state_roundtrip_without_iterations(ot):
    plan, g = make_plan(ot, (32, 24, 3), RGB, 6)
    f0, f1 = random_pair(g, 5)
    st = _random_state(g, 6)
    xp = f32(pack_path(g, st.m, st.f))
    bp = f32(pack_dual(g, st.bm, st.bf))
    bbp = f32(pack_dual(g, st.bbm, st.bbf))
    plan.state_set(f32(f0), f32(f1), xp, bp, bbp)
    x, b, bb = plan.state_get()
    assert np.array_equal(x, xp) and np.array_equal(b, bp)
    assert rel(bb, bbp) <= 1e-6


def _solve_both(ot, n, bc, P, iters, f0, f1):
    plan, g = make_plan(ot, n, bc, P)
    stats = plan.solve(f32(f0), f32(f1), iters)
    path = plan.path()
    st, infos, scale = o.solve(g, f0.astype(np.float64), f1.astype(np.float64), iters, SIG, TAU, with_dual=True)
    return plan, g, stats, path, st, infos, scale


def _check_dual(stats, info, scale):
    """The dual value of the last check (FP64 sums of compensated per-thread partials) against the
    oracle's, and the primal-dual gap formed from both sides' energy and dual value."""
    D = info.dual * scale
    assert abs(stats.dual_value - D) <= 1e-3 * abs(D)
    gap = abs(info.energy - info.dual) / max(abs(info.energy), abs(info.dual))
    assert abs(stats.gap - gap) <= 2e-3 + 1e-2 * gap


def test_full_solve_rgb_32x32x3x16_500_iterations(ot):
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(32, 32, 8, 0)
    plan, g, stats, path, st, infos, scale = _solve_both(ot, (32, 32, 3), RGB, 16, 500, f0, f1)
    assert stats.iterations == 500
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    for k in range(3):
        assert rel(path["m"][k][0], st.m[k] * scale) <= 1e-3
    assert abs(stats.energy - infos[-1].energy * scale) <= 1e-3 * infos[-1].energy * scale
    assert abs(stats.residual - infos[-1].residual) <= 1e-2 * infos[-1].residual + 1e-7
    assert stats.mass_drift <= 1e-5
    _check_dual(stats, infos[-1], scale)


def test_full_solve_periodic_xy_24x20x3x8(ot):
    """A torus image (periodic x, y and colour): 300 iterations against the oracle."""
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(24, 20, 4, 5)
    bc = ("periodic", "periodic", "periodic")
    plan, g, stats, path, st, infos, scale = _solve_both(ot, (24, 20, 3), bc, 8, 300, f0, f1)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    for k in range(3):
        assert rel(path["m"][k][0], st.m[k] * scale) <= 1e-3
    assert abs(stats.energy - infos[-1].energy * scale) <= 1e-3 * infos[-1].energy * scale
    assert stats.mass_drift <= 1e-5


def test_full_solve_periodic_xy_64x32x3x8(ot):
    """Periodic x, y and colour on power-of-two axes (the FFT real-Fourier transforms): 300 iterations
    against the oracle."""
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(64, 32, 4, 6)
    bc = ("periodic", "periodic", "periodic")
    plan, g, stats, path, st, infos, scale = _solve_both(ot, (64, 32, 3), bc, 8, 300, f0, f1)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    for k in range(3):
        assert rel(path["m"][k][0], st.m[k] * scale) <= 1e-3
    assert stats.mass_drift <= 1e-5


def test_full_solve_radix3_96x96x3x4(ot):
    """Sides of 3 * 2^k take the FFT path with a radix-3 step (96 = 16 * 6): 300 iterations against the
    oracle."""
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(96, 96, 6, 7)
    plan, g, stats, path, st, infos, scale = _solve_both(ot, (96, 96, 3), RGB, 4, 300, f0, f1)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    for k in range(3):
        assert rel(path["m"][k][0], st.m[k] * scale) <= 1e-3
    assert stats.mass_drift <= 1e-5


def test_full_solve_hue_360x64(ot):
    from paper_1501_04840_gb300 import synth
    h0, h1 = synth.hue_pair(360, 0)
    plan, g, stats, path, st, infos, scale = _solve_both(ot, (360,), ("periodic",), 64, 300, h0, h1)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    # m is unique only up to N(S_M) at the solution (section 2, Theorem 1); the
    # iterates from the same start coincide, and so does u = S_M m
    assert rel(path["m"][0][0], st.m[0] * scale) <= 1e-3
    u_gpu = o.S_M(g, [path["m"][0][0].astype(np.float64)])[0]
    assert rel(u_gpu, o.S_M(g, st.m)[0] * scale) <= 1e-3
    assert stats.mass_drift <= 1e-5
    _check_dual(stats, infos[-1], scale)


def test_batch_equals_single_problems(ot):
    from paper_1501_04840_gb300 import synth
    pairs = [synth.rgb_pair(48, 32, 8, s) for s in range(3)]
    f0 = np.stack([p[0] for p in pairs])
    f1 = np.stack([p[1] for p in pairs])
    g = ot.grid((48, 32, 3), RGB, 9, sigma=SIG, tau=TAU)
    plan = ot.Plan(g, batch=3)
    plan.solve(f32(f0), f32(f1), 40)
    pb = plan.path()
    for s in range(3):
        single = ot.Plan(ot.grid((48, 32, 3), RGB, 9, sigma=SIG, tau=TAU))
        single.solve(f32(pairs[s][0]), f32(pairs[s][1]), 40)
        ps = single.path()
        assert rel(pb["f"][s], ps["f"][0]) <= 1e-6
        for k in range(3):
            assert rel(pb["m"][k][s], ps["m"][k][0]) <= 1e-6


def test_input_validation(ot):
    plan, g = make_plan(ot, (32, 32, 3), RGB, 8)
    f0, f1 = random_pair(g, 7)
    bad = f0.copy()
    bad[0, 0, 0] = -1e-3
    with pytest.raises(ot.OTError) as ei:
        plan.solve(f32(bad), f32(f1), 5)
    assert ei.value.status == 2
    with pytest.raises(ot.OTError) as ei:
        plan.solve(f32(f0), f32(f1 * 1.01), 5)
    assert ei.value.status == 2
    nan = f0.copy()
    nan[1, 2, 3] = np.nan
    with pytest.raises(ot.OTError) as ei:
        plan.solve(f32(nan), f32(f1), 5)
    assert ei.value.status == 2
    # the plan still works afterwards
    st = plan.solve(f32(f0), f32(f1), 5)
    assert st.iterations == 5


@pytest.mark.parametrize("n,P", [((64, 64, 3), 16), ((128, 96, 3), 17), ((64, 48), 8)])
def test_staged_and_plain_update_kernels_agree(ot, n, P, monkeypatch):
    """The update kernel that stages its planes with bulk tensor copies does the same arithmetic as the
    plain-load one (DYNOT_UPDATE_KERNEL=plain); the compiler may contract a few products into fused
    multiply-adds differently, so seven iterations from the same random state agree to float32 rounding,
    amplified by the projection's correction A^T phi as in the parity bound (1e-5 relative), not bit for
    bit."""
    bc = RGB if len(n) == 3 else ("neumann", "neumann")
    g = oracle_grid(n, bc, P)
    f0, f1 = random_pair(g, 21)
    st = _random_state(g, 22, smooth=True)
    args = (f32(f0), f32(f1), f32(pack_path(g, st.m, st.f)), f32(pack_dual(g, st.bm, st.bf)),
            f32(pack_dual(g, st.bbm, st.bbf)))
    out = []
    for kind in ("staged", "plain"):
        if kind == "plain":
            monkeypatch.setenv("DYNOT_UPDATE_KERNEL", "plain")
        plan = ot.Plan(ot.grid(n, bc, P, sigma=SIG, tau=TAU))
        plan.state_set(*args)
        plan.iterate(7)
        out.append(plan.state_get())
        plan.close()
    for a, b in zip(out[0], out[1]):
        assert rel(a, b) <= 1e-5


@pytest.mark.parametrize("n,bc,P,precision", [((64, 64, 3), RGB, 16, 0), ((96, 64, 3), RGB, 12, 0),
                                                ((48, 40, 3), ("periodic", "neumann", "periodic"), 9, 0),
                                                ((64, 64, 3), RGB, 16, 2)])
def test_split_xt_passes_match_oracle(ot, n, bc, P, precision, monkeypatch):
    """The split x/t passes (r, the x transform of row blocks and the t transform of column strips in
    separate launches), which grids whose (t, x) plane exceeds shared memory take (the FP64 plan at
    512 x 512 x 3 x 64), selected here with DYNOT_SPLIT_XT=1: one iteration against the oracle with the
    bound of the fused passes (FP32), and to 1e-9 in FP64."""
    monkeypatch.setenv("DYNOT_SPLIT_XT", "1")
    g = oracle_grid(n, bc, P)
    plan = ot.Plan(ot.grid(n, bc, P, sigma=SIG, tau=TAU, precision=precision))
    f0, f1 = random_pair(g, 31)
    st = _random_state(g, 32, smooth=True)
    plan.state_set(f32(f0), f32(f1), f32(pack_path(g, st.m, st.f)), f32(pack_dual(g, st.bm, st.bf)),
                   f32(pack_dual(g, st.bbm, st.bbf)))
    plan.iterate(1)
    x, b, _ = plan.state_get()
    new, _ = o.pdhg_step(g, st, f0, f1, SIG, TAU)
    xo, bo = pack_path(g, new.m, new.f), pack_dual(g, new.bm, new.bf)
    tol = 1e-6 if precision == 2 else _step_tolerance(g, st, f0, f1)
    assert rel(x, xo) <= tol and rel(b, bo) <= tol


@pytest.mark.parametrize("bins,P,batch,smooth", [(360, 64, 8, False), (101, 32, 16, True), (720, 16, 40, False)])
def test_hue_batch_dft_product_matches_oracle(ot, bins, P, batch, smooth):
    """Hue plans of at least 512 rows (batch x P) run the real DFT along the bins as one dense matrix product
    over all rows: one iteration of every problem from its own random state against the oracle, with the
    bound of the single-problem tests."""
    g = oracle_grid((bins,), ("periodic",), P)
    plan = ot.Plan(ot.grid((bins,), ("periodic",), P, sigma=SIG, tau=TAU), batch=batch)
    pairs = [random_pair(g, 40 + i) for i in range(batch)]
    states = [_random_state(g, 60 + i, smooth) for i in range(batch)]
    cat = lambda parts: f32(np.concatenate([np.asarray(p, np.float64).ravel() for p in parts]))
    plan.state_set(cat([p[0] for p in pairs]), cat([p[1] for p in pairs]),
                   cat([pack_path(g, st.m, st.f) for st in states]), cat([pack_dual(g, st.bm, st.bf) for st in states]),
                   cat([pack_dual(g, st.bbm, st.bbf) for st in states]))
    plan.iterate(1)
    x, _, _ = plan.state_get()
    x = x.reshape(batch, -1)
    for i in range(batch):
        f0, f1 = pairs[i]
        new, _ = o.pdhg_step(g, states[i], f0, f1, SIG, TAU)
        assert rel(x[i], pack_path(g, new.m, new.f)) <= _step_tolerance(g, states[i], f0, f1)


def test_hue_batch_row_update_matches_cell_update(ot, monkeypatch):
    """A hue plan of 8 or more problems updates its plain iterations with the tiled kernel, the problems as
    its rows; DYNOT_UPDATE_KERNEL=plain keeps the cell-by-cell kernel.  Seven iterations (six plain, one
    check) from the same random states agree to float32 rounding (1e-5, as for the RGB update kernels)."""
    bins, P, batch = 101, 20, 12
    g = oracle_grid((bins,), ("periodic",), P)
    pairs = [random_pair(g, 80 + i) for i in range(batch)]
    states = [_random_state(g, 90 + i, True) for i in range(batch)]
    cat = lambda parts: f32(np.concatenate([np.asarray(p, np.float64).ravel() for p in parts]))
    args = (cat([p[0] for p in pairs]), cat([p[1] for p in pairs]),
            cat([pack_path(g, st.m, st.f) for st in states]), cat([pack_dual(g, st.bm, st.bf) for st in states]),
            cat([pack_dual(g, st.bbm, st.bbf) for st in states]))
    out = []
    for kind in ("rows", "plain"):
        if kind == "plain":
            monkeypatch.setenv("DYNOT_UPDATE_KERNEL", "plain")
        plan = ot.Plan(ot.grid((bins,), ("periodic",), P, sigma=SIG, tau=TAU), batch=batch)
        plan.state_set(*args)
        plan.iterate(7)
        out.append(plan.state_get())
        plan.close()
    for a, b in zip(out[0], out[1]):
        assert rel(a, b) <= 1e-5


@pytest.mark.parametrize("where", ["dual", "path"])
def test_non_finite_state_is_reported(ot, where):
    """The detector of non-finite residuals: a NaN planted on the host in the dual (or an Inf in the
    path) through ot_state_set makes the residual of the next check non-finite, and ot_iterate returns
    OT_ENUMERIC.  Nothing faults on the device, and the plan stays usable: a finite state set
    afterwards iterates normally."""
    plan, g = make_plan(ot, (32, 24, 3), RGB, 6)
    f0, f1 = random_pair(g, 11)
    st = _random_state(g, 12)
    xp = f32(pack_path(g, st.m, st.f))
    bp = f32(pack_dual(g, st.bm, st.bf))
    bad_x, bad_b = xp.copy(), bp.copy()
    if where == "dual":
        bad_b[bad_b.size // 3] = np.nan
    else:
        bad_x[bad_x.size // 2] = np.inf
    plan.state_set(f32(f0), f32(f1), bad_x, bad_b)
    with pytest.raises(ot.OTError) as ei:
        plan.iterate(3)
    assert ei.value.status == ot.OT_ENUMERIC
    plan.state_set(f32(f0), f32(f1), xp, bp)
    out = plan.iterate(3)
    assert out.iterations == 3 and np.isfinite(out.residual)


def test_tolerance_stops_early_and_reports(ot):
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(32, 32, 8, 0)
    plan, g = make_plan(ot, (32, 32, 3), RGB, 16)
    st = plan.solve(f32(f0), f32(f1), 2000, tol=1e-4, check_every=10)
    assert st.converged and st.residual <= 1e-4 and st.iterations % 10 == 0 and st.iterations < 2000
    st2 = plan.solve(f32(f0), f32(f1), 20, tol=1e-12)
    assert not st2.converged and st2.iterations == 20


def test_fp64_plan_matches_oracle_tightly(ot):
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(32, 32, 8, 0)
    plan, g = make_plan(ot, (32, 32, 3), RGB, 16, precision=2)
    plan.solve(f32(f0), f32(f1), 200)
    path = plan.path()
    st, infos, scale = o.solve(g, f0.astype(np.float64), f1.astype(np.float64), 200, SIG, TAU)
    assert rel(path["f"][0], st.f * scale) <= 1e-6   # limited by the float32 path output


def test_warm_start_matches_oracle(ot):
    """init_path: x0 = init (caller units), b = bbar = 0, as the oracle started from that state."""
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(32, 32, 8, 1)
    plan, g = make_plan(ot, (32, 32, 3), RGB, 16)
    f0d, f1d = f0.astype(np.float64), f1.astype(np.float64)
    # an initial path from the oracle (100 cold iterations), in caller units
    st0, _, scale = o.solve(g, f0d, f1d, 100, SIG, TAU)
    init = pack_path(g, [a * scale for a in st0.m], st0.f * scale).astype(np.float32)
    stats = plan.solve(f32(f0), f32(f1), 50, init=init)
    path = plan.path()
    start = o.State.zeros(g)
    m_init, f_init = unpack_path(g, init.astype(np.float64))
    start.m = [a / scale for a in m_init]
    start.f = f_init / scale
    st, infos, _ = o.solve(g, f0d, f1d, 50, SIG, TAU, state=start)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    assert abs(stats.energy - infos[-1].energy * scale) <= 1e-3 * infos[-1].energy * scale


# ---- the benchmark's size and launch configuration --------------------------

def test_full_size_one_iteration_matches_oracle(ot):
    n, P = (256, 256, 3), 32
    plan, g = make_plan(ot, n, RGB, P)
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(256, 256, 32, 0)
    f0 = f0.astype(np.float64)
    f1 = f1.astype(np.float64)
    st = _random_state(g, 8, smooth=True)
    plan.state_set(f32(f0), f32(f1), f32(pack_path(g, st.m, st.f)), f32(pack_dual(g, st.bm, st.bf)),
                   f32(pack_dual(g, st.bbm, st.bbf)))
    plan.iterate(1)
    x, b, bb = plan.state_get()
    new, _ = o.pdhg_step(g, st, f0, f1, SIG, TAU)
    tol = _step_tolerance(g, st, f0, f1)
    m, f = unpack_path(g, x.astype(np.float64))
    assert rel(f, new.f) <= tol
    for k in range(3):
        assert rel(m[k], new.m[k]) <= tol
    bm, bf = unpack_dual(g, b.astype(np.float64))
    assert rel(bf, new.bf) <= tol


def test_full_size_solve_first_iterations_and_invariants(ot):
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(256, 256, 32, 0)
    plan, g = make_plan(ot, (256, 256, 3), RGB, 32)
    stats = plan.solve(f32(f0), f32(f1), 4)
    path = plan.path()
    st, infos, scale = o.solve(g, f0.astype(np.float64), f1.astype(np.float64), 4, SIG, TAU)
    assert rel(path["f"][0], st.f * scale) <= 1e-4
    assert stats.mass_drift <= 1e-5
    # mass of every interior time slice equals the mass of f0 (section 2, C_d)
    sums = path["f"][0].reshape(g.P - 1, -1).astype(np.float64).sum(axis=1)
    np.testing.assert_allclose(sums, f0.astype(np.float64).sum(), rtol=1e-5)


def test_profile_reports_every_kernel(ot):
    plan, g = make_plan(ot, (64, 64, 3), RGB, 16)
    f0, f1 = random_pair(g, 9)
    plan.solve(f32(f0), f32(f1), 2)
    ms = plan.profile(4)
    assert set(ms) == {"rhs_fwd_xt", "solve_yc", "inv_xt", "update", "iteration"}
    assert all(v > 0 for v in ms.values())


@pytest.mark.parametrize("colour_bc", ["periodic", "neumann"])
def test_fig1_red_to_blue_matches_oracle(ot, colour_bc):
    """Fig. 1's red -> blue Gaussian on the GPU with periodic and with Neumann colour: the path after
    600 iterations against the oracle, and the green share at t = 1/2 (small for periodic colour,
    most of the mass for Neumann colour)."""
    from test_oracle_solve import _fig1_pair
    n, P = 12, 8
    f0, f1 = _fig1_pair(n)
    bc = ("neumann", "neumann", colour_bc)
    plan, g = make_plan(ot, (n, n, 3), bc, P)
    plan.solve(f32(f0), f32(f1), 600)
    path = plan.path()
    st, _, sc = o.solve(g, f32(f0).astype(np.float64), f32(f1).astype(np.float64), 600, SIG, TAU)
    assert rel(path["f"][0], st.f * sc) <= 1e-3
    mid = path["f"][0][P // 2 - 1].astype(np.float64)
    green = mid[1].sum() / mid.sum()
    ref = (st.f[P // 2 - 1] * sc)[1].sum() / (st.f[P // 2 - 1] * sc).sum()
    assert abs(green - ref) <= 1e-3
    assert (green < 0.15) if colour_bc == "periodic" else (green > 0.5)
