"""Mixed-size batches (ot_batch_*) against single plans and the oracle (GPU).

Every problem of a batch follows Algorithm 1 exactly as a plan of its own
does, so its path after a fixed number of iterations equals the single-plan
path; shapes that repeat share one batched plan."""
import numpy as np
import pytest

import oracle as o
from _helpers import f32, oracle_grid, rel

pytestmark = pytest.mark.gpu

SIG, TAU = 0.3, 0.99 / 0.3
RGB = ("neumann", "neumann", "periodic")


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


def _problems():
    from paper_1501_04840_gb300 import synth
    probs = [((32, 32, 3), RGB, 8, synth.rgb_pair(32, 32, 8, 0)),
             ((48, 40, 3), RGB, 9, synth.rgb_pair(48, 40, 8, 1)),
             ((32, 32, 3), RGB, 8, synth.rgb_pair(32, 32, 8, 2)),
             ((64,), ("periodic",), 16, synth.hue_pair(64, 0)),
             ((101,), ("periodic",), 20, synth.hue_pair(101, 1))]
    return probs


def test_batch_equals_single_plans(ot):
    probs = _problems()
    grids = [ot.grid(n, bc, P, sigma=SIG, tau=TAU) for n, bc, P, _ in probs]
    batch = ot.Batch(grids)
    assert batch.groups == 4          # the two 32x32x3x8 problems share a plan
    stats = batch.solve([f32(p[3][0]) for p in probs], [f32(p[3][1]) for p in probs], 41, check_every=10)
    assert all(s.iterations == 41 for s in stats)
    for i, (n, bc, P, (f0, f1)) in enumerate(probs):
        plan = ot.Plan(ot.grid(n, bc, P, sigma=SIG, tau=TAU))
        st = plan.solve(f32(f0), f32(f1), 41, check_every=10)
        ps = plan.path()
        pb = batch.path(i)
        assert rel(pb["f"], ps["f"][0]) <= 1e-6
        for k in range(len(n)):
            assert rel(pb["m"][k], ps["m"][k][0]) <= 1e-6
        assert stats[i].residual == pytest.approx(st.residual, rel=1e-6)


def test_batch_matches_oracle_and_stops_at_tolerance(ot):
    probs = _problems()
    grids = [ot.grid(n, bc, P, sigma=SIG, tau=TAU) for n, bc, P, _ in probs]
    batch = ot.Batch(grids)
    stats = batch.solve([f32(p[3][0]) for p in probs], [f32(p[3][1]) for p in probs], 3000, tol=1e-4,
                        check_every=10)
    assert all(s.converged and s.residual <= 1e-4 for s in stats)
    for i, (n, bc, P, (f0, f1)) in enumerate(probs):
        g = oracle_grid(n, bc, P)
        st, infos, scale = o.solve(g, f0.astype(np.float64), f1.astype(np.float64), stats[i].iterations, SIG, TAU)
        assert rel(batch.path(i)["f"], st.f * scale) <= 1e-3
        assert stats[i].mass_drift <= 1e-5


def test_converged_problems_retire(ot):
    """Each problem stops at the first check where its own residual meets tol: its iteration count, its
    path and its residual equal those of a single plan solved to the same tolerance, so the batch does no
    more cell-iterations than the problems solved one by one."""
    probs = _problems()
    grids = [ot.grid(n, bc, P, sigma=SIG, tau=TAU) for n, bc, P, _ in probs]
    batch = ot.Batch(grids)
    stats = batch.solve([f32(p[3][0]) for p in probs], [f32(p[3][1]) for p in probs], 3000, tol=1e-4,
                        check_every=10)
    its = [s.iterations for s in stats]
    assert len(set(its)) > 1      # the problems converge at different checks
    for i, (n, bc, P, (f0, f1)) in enumerate(probs):
        plan = ot.Plan(ot.grid(n, bc, P, sigma=SIG, tau=TAU))
        st = plan.solve(f32(f0), f32(f1), 3000, tol=1e-4, check_every=10)
        assert st.converged and stats[i].iterations == st.iterations
        assert stats[i].residual == pytest.approx(st.residual, rel=1e-6)
        ps, pb = plan.path(), batch.path(i)
        assert rel(pb["f"], ps["f"][0]) <= 1e-6


def test_plans_sharing_kernels_coexist(ot):
    """A later plan of the same kernels must not lower an earlier plan's shared-memory limit."""
    from paper_1501_04840_gb300 import synth
    shapes = [(688, 47), (64, 47), (256, 192, 32), (64, 64, 32)]
    plans, pairs = [], []
    for sh in shapes:
        if len(sh) == 2:
            plans.append(ot.Plan(ot.hue_grid(sh[0], sh[1])))
            pairs.append(synth.hue_pair(sh[0], 0))
        else:
            plans.append(ot.Plan(ot.rgb_grid(sh[0], sh[1], sh[2])))
            pairs.append(synth.rgb_pair(sh[0], sh[1], 8, 0))
    for pl, (f0, f1) in zip(plans, pairs):
        st = pl.solve(f32(f0), f32(f1), 20, check_every=10)
        assert st.iterations == 20 and np.isfinite(st.residual)
