"""Planted mistakes in the oracle, on the CPU.

Each mutant rewrites one expression of one oracle function: a dropped term or
factor, a flipped sign, a wrong neighbour index or operand, a wrong
normalisation. The pins of tests/test_oracle_*.py must reject every one of them.
This checks the pins rather than the oracle: a plausible slip anywhere in the
oracle's operators (section 2), projection (section 3, step 1), prox (section 3,
step 2) or iteration (Algorithm 1) fails at least one pin.
"""
import inspect
import textwrap

import numpy as np
import pytest

import oracle
import oracle.dynot as od
import oracle.huepipe as ohp
import oracle.unet as ou
import test_oracle_huepipe as thp
import test_oracle_operators as ops
import test_oracle_projection as proj
import test_oracle_prox as prx
import test_oracle_solve as slv
import test_oracle_unet as tun

# (function, expression as written in oracle/dynot.py, planted mistake)
MUTANTS = [
    ("S_M", "out.append(0.5 * (left + right))", "out.append(left + right)"),
    ("S_M_T", "np.roll(uk, 1, axis=ax) + uk", "np.roll(uk, -1, axis=ax) + uk"),
    ("S_F_T", "0.5 * (v[:-1] + v[1:])", "0.5 * (v[:-1] - v[1:])"),
    ("f_b_plus", "out[-1] += 0.5 * f1", "out[-1] += 0.5 * f0"),
    ("f_b_minus", "out[-1] -= g.P * f1", "out[-1] += g.P * f1"),
    ("D_M", "(np.roll(mk, -1, axis=ax) - mk)", "(mk - np.roll(mk, -1, axis=ax))"),
    ("D_F", "g.P * (F[1:] - F[:-1])", "(F[1:] - F[:-1])"),
    ("A_T", "ft = -g.P * (phi[1:] - phi[:-1])", "ft = g.P * (phi[1:] - phi[:-1])"),
    ("eigenvalues", "g.P ** 2 * 4.0 * np.sin", "g.P * 4.0 * np.sin"),
    ("eigenvalues", "q = 4.0 * np.sin(j * np.pi / g.n[k]) ** 2", "q = 4.0 * np.sin(j * np.pi / (2 * g.n[k])) ** 2"),
    ("poisson_pinv", 'h = scipy.fft.dct(r, type=2, norm="ortho", axis=0)', "h = scipy.fft.dct(r, type=2, axis=0)"),
    ("project", "r = A(g, am, af) - f_b_minus(g, f0, f1)", "r = A(g, am, af) + f_b_minus(g, f0, f1)"),
    ("prox_J", "pos = af + 0.5 * sigma * s2 > 0", "pos = af > 0"),
    ("prox_J", "np.where(pos, sigma * v * a / (1.0 + sigma * v), 0.0)", "np.where(pos, v * a / (1.0 + sigma * v), 0.0)"),
    ("J_energy", "out[pos] = s2[pos] / (2.0 * v[pos])", "out[pos] = s2[pos] / v[pos]"),
    ("pdhg_step", "am = [st.m[k] - tau * sigma * km[k]", "am = [st.m[k] + tau * sigma * km[k]"),
    ("pdhg_step", "a_f = sf + fbp + st.bf", "a_f = sf + st.bf"),
    ("pdhg_step", "bf = a_f - v", "bf = a_f + v"),
    ("pdhg_step", "bbf = bf + theta * (bf - st.bf)", "bbf = bf + theta * (st.bf - bf)"),
    ("dual_value", "np.sum(bf * (sf + fbp))", "np.sum(bf * sf)"),
    ("dual_value", "return sigma * tot / g.ncells", "return tot / g.ncells"),
    ("min_norm_path", "m, f, _ = project(g, zm, np.zeros(g.f_shape), f0, f1)", "m, f = zm, np.zeros(g.f_shape)"),
]


# the network layers (oracle/unet.py) and the hue pipeline (oracle/huepipe.py)
UNET_MUTANTS = [
    ("conv3d", "win = xp[:, 1 + dt:1 + dt + T, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X, :]",
     "win = xp[:, 1 - dt:1 - dt + T, 1 - dy:1 - dy + Y, 1 - dx:1 - dx + X, :]"),
    ("conv3d_dgrad", "win = gp[:, 1 - dt:1 - dt + T, 1 - ddy:1 - ddy + Y, 1 - dxx:1 - dxx + X, :]",
     "win = gp[:, 1 + dt:1 + dt + T, 1 + ddy:1 + ddy + Y, 1 + dxx:1 + dxx + X, :]"),
    ("conv3d_wgrad", 'dw[:, k, :] = np.einsum("ntyxo,ntyxc->oc", g, win)', 'dw[:, 26 - k, :] = np.einsum("ntyxo,ntyxc->oc", g, win)'),
    ("pool_backward", "axis=3) * 0.25", "axis=3)"),
    ("upsample_backward", ".sum(axis=(3, 5))", ".mean(axis=(3, 5))"),
    ("relu_backward", "np.asarray(y) > 0", "np.asarray(y) >= 0"),
    ("mse", "2.0 * d / d.size", "d / d.size"),
    ("adamw", "p * (1 - lr * wd)", "p * (1 - wd)"),
    ("adamw", "(m / (1 - b1 ** step))", "m"),
    ("round_bf16", "(u + 0x7FFF + ((u >> 16) & 1))", "(u + 0x8000)"),
]
HUE_MUTANTS = [
    ("rgb_to_hsv", "(b - r) / safe + 2.0", "(r - b) / safe + 2.0"),
    ("hsv_to_rgb", "np.choose(i, [t, v, v, q, p, p])", "np.choose(i, [t, v, q, v, p, p])"),
    ("hue_bin", "np.floor(np.asarray(h, np.float64) * bins)", "np.round(np.asarray(h, np.float64) * bins)"),
    ("exact_counts", "np.lexsort((np.arange(len(x)), -rem))", "np.lexsort((np.arange(len(x)), rem))"),
    ("target_hues", "(q - C[b] + 0.5) / counts[b]", "(q - C[b]) / counts[b]"),
    ("circular_sq", "d = np.minimum(d, 1.0 - d)", "d = d"),
    ("best_shift", "int(np.argmin(all_shift_costs(x, y)))", "int(np.argmin(all_shift_costs(x, y)[:len(x) // 2]))"),
    ("strict_order", "np.lexsort((np.arange(len(q)), q.astype(np.uint64)))",
     "np.lexsort((q.astype(np.uint64), np.arange(len(q))))"),
]


def _mutant(name, old, new, mod=od):
    src = textwrap.dedent(inspect.getsource(getattr(mod, name)))
    assert src.count(old) == 1, "the expression to mutate must occur once in %s" % name
    scope = {}
    exec(compile(src.replace(old, new), "<mutant of %s>" % name, "exec"), mod.__dict__, scope)
    return scope[name]


def _pins():
    """The oracle's pins, cheapest first (a few seconds in all when nothing fails)."""
    for g in ops.GRIDS:
        ops.test_operators_match_dense(g)
    for g in ops.GRIDS[:4]:
        ops.test_boundary_vectors(g)
    ops.test_continuity_is_forward_difference_in_time()
    ops.test_periodic_even_null_space_of_S_M()
    for g in proj.GRIDS:
        proj.test_eigenvalues_match_dense(g)
        proj.test_projection_matches_pinv_and_lstsq(g)
        proj.test_poisson_pinv_matches_dense(g)
    proj.test_projection_preserves_mass_per_time()
    for case in prx.CASES:
        prx.test_prox_optimality_and_cubic(*case)
    prx.test_prox_zero_case()
    slv.test_mass_per_time_slice_every_iteration()
    slv.test_colour_shift_equivariance()
    slv.test_time_reversal_equivariance()
    slv.test_remark1_nonunique_zero_energy()
    slv.test_equal_endpoints_give_zero_energy()
    slv.test_quantile_closed_form_1d_neumann()
    slv.test_primal_dual_gap_vanishes_at_convergence()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=["%s:%d" % (m[0], i) for i, m in enumerate(MUTANTS)])
def test_pins_reject_planted_mistake(monkeypatch, name, old, new):
    fn = _mutant(name, old, new)
    monkeypatch.setattr(od, name, fn)        # calls inside the oracle
    monkeypatch.setattr(oracle, name, fn)    # calls from the pins
    with pytest.raises((AssertionError, FloatingPointError, ValueError)), np.errstate(all="ignore"):
        _pins()


def _unet_pins():
    tun.test_conv3d_matches_scipy_correlate()
    tun.test_conv3d_gradients_by_finite_differences()
    tun.test_pool_upsample_adjoint_pairs()
    tun.test_mse_gradient()
    tun.test_adamw_closed_forms()
    tun.test_round_bf16_against_the_format()
    tun.test_unet_gradients_by_finite_differences()


def _hue_pins():
    thp.test_hsv_against_colorsys()
    thp.test_exact_counts_by_hand()
    thp.test_target_hues_by_hand()
    thp.test_specification_is_exact()
    thp.test_specification_to_the_source_histogram_keeps_every_bin()
    for k in (1, 3, 58, 59):
        thp.test_specification_to_a_slightly_rotated_histogram_rotates_every_pixel(k)
    for seed in range(3):
        thp.test_best_cyclic_shift_is_the_optimal_assignment(seed)
    for n, k in ((4096, 1), (4096, -3)):
        thp.test_rotated_bump_is_cut_at_the_rotation(n, k)


@pytest.mark.parametrize("name,old,new", UNET_MUTANTS, ids=["%s:%d" % (m[0], i) for i, m in enumerate(UNET_MUTANTS)])
def test_network_pins_reject_planted_mistake(monkeypatch, name, old, new):
    monkeypatch.setattr(ou, name, _mutant(name, old, new, ou))
    with pytest.raises((AssertionError, FloatingPointError, ValueError)), np.errstate(all="ignore"):
        _unet_pins()


@pytest.mark.parametrize("name,old,new", HUE_MUTANTS, ids=["%s:%d" % (m[0], i) for i, m in enumerate(HUE_MUTANTS)])
def test_hue_pipeline_pins_reject_planted_mistake(monkeypatch, name, old, new):
    monkeypatch.setattr(ohp, name, _mutant(name, old, new, ohp))
    with pytest.raises((AssertionError, FloatingPointError, ValueError)), np.errstate(all="ignore"):
        _hue_pins()
