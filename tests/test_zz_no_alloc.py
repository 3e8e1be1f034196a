"""ot_hue_project_noalloc against ot_project (GPU, through the C ABI).

The no-allocation entry point serves callers that cannot allocate device
memory; it must give the same projection as a hue plan, call after call (the
fixed working array keeps the previous call's data, which must not leak into
the next result)."""
import ctypes

import numpy as np
import pytest

from _helpers import EPS32, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_04840_gb300 import _build
    _build.build()
    import paper_1501_04840_gb300 as p
    lib = p.load_library()
    fn = lib.ot_hue_project_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double] + [ctypes.c_void_p] * 6
    fn.restype = ctypes.c_int
    return torch, p, lib, fn


def _inputs(bins, P, batch, seed):
    rng = np.random.default_rng(seed)
    f0 = (rng.random((batch, bins)) + 0.2).astype(np.float32)
    f1 = (rng.random((batch, bins)) + 0.2).astype(np.float32)
    f1 = (f1 * (f0.sum(1, keepdims=True) / f1.sum(1, keepdims=True))).astype(np.float32)
    per = P * bins + (P - 1) * bins
    a = rng.standard_normal((batch, per)).astype(np.float32)
    return f0, f1, a


@pytest.mark.parametrize("bins,P,batch", [(360, 64, 2), (101, 20, 3), (4096, 64, 1)])
def test_noalloc_matches_plan_projection_twice(env, bins, P, batch):
    torch, p, lib, fn = env
    plan = p.Plan(p.hue_grid(bins, P), batch=batch)
    for call in range(2):   # two calls in a row with different data
        f0, f1, a = _inputs(bins, P, batch, seed=10 * call + bins)
        x_ref, phi_ref = plan.project(f0, f1, a.ravel(), with_phi=True)
        dev = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
        d0, d1, da = dev(f0), dev(f1), dev(a)
        dx = torch.empty_like(da)
        dphi = torch.empty((batch, P, bins), dtype=torch.float32, device="cuda")
        st = fn(bins, P, batch, 0.0, d0.data_ptr(), d1.data_ptr(), da.data_ptr(), dx.data_ptr(),
                dphi.data_ptr(), None)
        assert st == 0, lib.ot_last_error()
        torch.cuda.synchronize()   # the call only queues its kernel
        x = dx.cpu().numpy().ravel()
        phi = dphi.cpu().numpy().ravel()
        # both sides sum the dense real DFT over the bins in float32, each with a rounding error of about
        # eps32 sqrt(bins) relative: 1e-5 up to about 1600 bins, 4 eps32 sqrt(bins) beyond
        assert rel(phi, phi_ref) <= max(1e-5, 4 * EPS32 * np.sqrt(bins))
        # x = a - A^T phi: the tolerance of the parity tests for this correction, plus the difference of
        # the two phi carried through A^T (||A^T d|| <= sqrt(lam_max) ||d||), which the dense float32
        # sums over thousands of bins make larger than the FFT-based transforms' ten epsilons
        lam_max = (2 * bins) ** 2 + (2 * P) ** 2
        kappa = np.sqrt(lam_max) * np.linalg.norm(phi_ref) / np.linalg.norm(x_ref)
        carried = np.sqrt(lam_max) * np.linalg.norm(phi.astype(np.float64) - phi_ref) / np.linalg.norm(x_ref)
        assert rel(x, x_ref) <= 1e-5 + 10 * EPS32 * kappa + 1.01 * carried


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, p, lib, fn = env
    d = torch.zeros(16, device="cuda")
    st = fn(720, 64, 100, 0.0, d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), None)
    assert st == 1 and b"scratch" in lib.ot_last_error()


def test_noalloc_rejects_a_bad_axis_scale(env):
    """axis_scale 0 means the default (bins); a negative, infinite or NaN one is an error, as ot_plan's
    validation makes it."""
    torch, p, lib, fn = env
    d = torch.zeros(2 * 64 * 8, device="cuda")
    for bad in (-1.0, float("nan"), float("inf")):
        st = fn(8, 4, 1, bad, d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), None)
        assert st == 1 and b"axis_scale" in lib.ot_last_error()
