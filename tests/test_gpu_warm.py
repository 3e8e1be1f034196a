"""Warm starts of Algorithm 1 (ot_solve_warm) and the warm-start network's
gradients, against the oracle (GPU)."""
import numpy as np
import pytest

import oracle as o
from oracle import unet
from _helpers import f32, oracle_grid, pack_path, rel, unpack_path

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


def _plan(ot, n=(32, 32, 3), P=16):
    return ot.Plan(ot.grid(n, RGB, P, sigma=SIG, tau=TAU)), oracle_grid(n, RGB, P)


def _pair_and_init(g, iters=100):
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(g.n[0], g.n[1], 8, 3)
    f0d, f1d = f0.astype(np.float64), f1.astype(np.float64)
    st0, _, scale = o.solve(g, f0d, f1d, iters, SIG, TAU)
    init = pack_path(g, [a * scale for a in st0.m], st0.f * scale).astype(np.float32)
    return f0, f1, init, scale


@pytest.mark.parametrize("dual,support", [(True, 0.0), (True, 0.3), (False, 0.0)])
def test_warm_start_matches_oracle(ot, dual, support):
    """x0 from an unfinished oracle run; the dual from the fixed-point formula (or zero)."""
    plan, g = _plan(ot)
    f0, f1, init, scale = _pair_and_init(g)
    stats = plan.solve_warm(f32(f0), f32(f1), init, 40, dual_init=dual, dual_support=support)
    path = plan.path()
    g0, g1, _ = o.normalise_pair(g, f0.astype(np.float64), f1.astype(np.float64))
    m_init, f_init = unpack_path(g, init.astype(np.float64))
    start = o.warm_state(g, [a / scale for a in m_init], f_init / scale, g0, g1, SIG, dual=dual, support=support)
    st, infos, _ = o.solve(g, f0.astype(np.float64), f1.astype(np.float64), 40, SIG, TAU, state=start)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    for k in range(3):
        assert rel(path["m"][k][0], st.m[k] * scale) <= 1e-3
    assert abs(stats.energy - infos[-1].energy * scale) <= 1e-3 * infos[-1].energy * scale
    assert abs(stats.residual - infos[-1].residual) <= 1e-2 * infos[-1].residual + 1e-6


def test_warm_start_with_given_dual_matches_oracle(ot):
    """x0 and b0 = bbar0 from an unfinished oracle run, passed through init_path / init_dual."""
    from _helpers import pack_dual
    plan, g = _plan(ot)
    from paper_1501_04840_gb300 import synth
    f0, f1 = synth.rgb_pair(32, 32, 8, 3)
    f0d, f1d = f0.astype(np.float64), f1.astype(np.float64)
    st0, _, scale = o.solve(g, f0d, f1d, 60, SIG, TAU)
    init = pack_path(g, [a * scale for a in st0.m], st0.f * scale).astype(np.float32)
    b0 = pack_dual(g, st0.bm, st0.bf).astype(np.float32)
    stats = plan.solve_warm(f32(f0), f32(f1), init, 40, init_dual=b0, dual_init=True)
    path = plan.path()
    start = o.State([a.copy() for a in st0.m], st0.f.copy(), [a.copy() for a in st0.bm], st0.bf.copy(),
                    [a.copy() for a in st0.bm], st0.bf.copy())
    st, infos, _ = o.solve(g, f0d, f1d, 40, SIG, TAU, state=start)
    assert rel(path["f"][0], st.f * scale) <= 1e-3
    for k in range(3):
        assert rel(path["m"][k][0], st.m[k] * scale) <= 1e-3
    assert abs(stats.residual - infos[-1].residual) <= 1e-2 * infos[-1].residual + 1e-6


def test_warm_without_dual_equals_init_path(ot):
    """ot_solve_warm with dual_init = 0 is ot_solve with init_path (same launches, same bits)."""
    plan, g = _plan(ot)
    f0, f1, init, _ = _pair_and_init(g, 30)
    plan.solve(f32(f0), f32(f1), 30, init=init)
    a = plan.path()
    plan.solve_warm(f32(f0), f32(f1), init, 30, dual_init=False)
    b = plan.path()
    assert np.array_equal(a["f"], b["f"]) and all(np.array_equal(x, y) for x, y in zip(a["m"], b["m"]))


def test_fallback_restarts_cold(ot):
    """A warm start whose first residual is above the threshold is dropped for the cold start."""
    plan, g = _plan(ot)
    f0, f1, init, _ = _pair_and_init(g, 5)
    st = plan.solve_warm(f32(f0), f32(f1), init, 60, dual_init=True, fallback_residual=1e-30, check_every=10)
    assert st.used_cold and st.iterations == 60
    warm = plan.path()
    plan.solve(f32(f0), f32(f1), 50, check_every=10)
    cold = plan.path()
    assert np.array_equal(warm["f"], cold["f"])
    st = plan.solve_warm(f32(f0), f32(f1), init, 20, dual_init=True, fallback_residual=1e30, check_every=10)
    assert not st.used_cold


def test_warm_start_from_converged_path_needs_few_iterations(ot):
    """With a density bounded away from zero the fixed-point dual of a converged path is the
    converged dual (grad J is defined everywhere), so the warm start sits at the fixed point."""
    from _helpers import random_pair
    plan, g = _plan(ot)
    a, b = random_pair(g, 21, floor=0.5)
    f0, f1 = f32(a), f32(b)
    cold = plan.solve(f0, f1, 20000, 1e-6, check_every=10)
    assert cold.converged
    x = plan.state_get()[0]                      # solver units, packed
    scale = 0.5 * (f0.astype(np.float64).sum() + f1.astype(np.float64).sum()) / f0.size
    init = (x.astype(np.float64) * scale).astype(np.float32)
    c4 = plan.solve(f0, f1, 20000, 1e-5, check_every=10)
    w4 = plan.solve_warm(f0, f1, init, 20000, 1e-5, dual_init=True, check_every=10)
    z4 = plan.solve_warm(f0, f1, init, 20000, 1e-5, dual_init=False, check_every=10)
    assert c4.converged and w4.converged and z4.converged
    print("iterations to 1e-5: cold %d, warm with dual %d, warm without dual %d" % (
        c4.iterations, w4.iterations, z4.iterations))
    assert w4.iterations == 10 < z4.iterations < c4.iterations


def test_unet_gradients_match_oracle(ot):
    """Forward and backward of a two-level U-Net on the GPU against the FP64 composition of
    oracle/unet.py with the same bf16 roundings (stored activations and activation gradients).
    What remains is fp32 against fp64 accumulation: rare one-ulp bf16 flips, well below 5e-3."""
    import torch
    from paper_1501_04840_gb300 import nn as K, warmstart as W
    from paper_1501_04840_gb300 import synth
    widths = (16, 32)
    net = W.UNet(widths, seed=3)
    # a larger head than the default so that every layer sees a real gradient
    p = net.p32.cpu().numpy()
    wo, nw, _, _ = net.off["head"]
    p[wo:wo + nw] = np.random.default_rng(4).standard_normal(nw) * 0.1
    net = W.UNet(widths, params=p)
    N, P, Y, X = 2, 4, 8, 12
    f0s, f1s = [], []
    for s in range(N):
        a, b = synth.rgb_pair(X, Y, 3, 10 + s)
        a, b = W.to_solver_units(a, b)
        f0s.append(a)
        f1s.append(b)
    f0 = torch.from_numpy(np.stack(f0s)).cuda()
    f1 = torch.from_numpy(np.stack(f1s)).cuda()
    B = net.buffers(N, P, Y, X, True)
    K.make_input(N, P, Y, X, f0, f1, B.inp)
    target = torch.from_numpy(np.random.default_rng(5).standard_normal((N, P, Y, X, W.CV)).astype(np.float32))
    target = target.to(torch.bfloat16).cuda()
    net.forward(B)
    net.g32.zero_()
    B.loss.zero_()
    net.backward(B, target)
    torch.cuda.synchronize()
    inp = B.inp.cpu().double().numpy()
    loss, out, grads = unet.unet_forward_backward(net.params_numpy(), widths, inp, target.cpu().double().numpy(),
                                                  W.CV, rnd=unet.round_bf16)
    assert abs(B.loss.item() - loss) <= 1e-3 * loss
    assert rel(B.out.cpu().double().numpy(), out) <= 5e-3
    got = net.grads_numpy()
    for name in grads:
        assert rel(got[name][0], grads[name][0]) <= 5e-3, name
        assert rel(got[name][1], grads[name][1]) <= 5e-3, name


def test_trained_network_beats_cold_start(ot):
    """The packaged U-Net (trained on 2000 solver-generated pairs at 128x128x3, P = 32) against the
    cold start on held-out pairs: fewer iterations and less wall time (inference included; median over the
    pairs) to residual 1e-4, and the same accuracy against a solve to 1e-6."""
    import os
    from paper_1501_04840_gb300 import warmstart as W
    if not os.path.exists(W.DEFAULT_WEIGHTS):
        pytest.skip("no trained weights in the package")
    net, meta = W.UNet.load(W.DEFAULT_WEIGHTS)
    ev = W.evaluate(net, list(range(1_000_000, 1_000_006)), 128, 32, 16, variants=(("net", "net", 0.0),))
    cold, warm = ev["cold"], ev["net"]
    print("cold %.1f it %.1f ms err %.3f | warm %.1f it %.1f ms err %.3f" % (
        cold["iters"]["mean"], cold["ms"]["mean"], cold["err"]["mean"], warm["iters"]["mean"], warm["ms"]["mean"],
        warm["err"]["mean"]))
    assert cold["all_converged"] and warm["all_converged"]
    assert warm["iters"]["mean"] <= 0.92 * cold["iters"]["mean"]
    # wall time by the median over the pairs, which a one-off stall of the process in one pair does not move
    assert warm["ms"]["p50"] < cold["ms"]["p50"]
    assert warm["err"]["mean"] <= cold["err"]["mean"] + 0.01
