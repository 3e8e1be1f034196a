"""ctypes binding of the C ABI in include/dynot.h (argument marshalling only).

Every numerical step runs in libdynot.so; this module only converts numpy
arrays and torch tensors to pointers and back.  Loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_size_t, c_void_p
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdynot.so")

OT_OK, OT_EINVAL, OT_EMASS, OT_ENOMEM, OT_ECUDA, OT_ETIMEOUT, OT_ENUMERIC, OT_ENOTCONV, OT_EUNSUPPORTED = range(9)
STATUS_NAMES = {0: "OT_OK", 1: "OT_EINVAL", 2: "OT_EMASS", 3: "OT_ENOMEM", 4: "OT_ECUDA", 5: "OT_ETIMEOUT",
                6: "OT_ENUMERIC", 7: "OT_ENOTCONV", 8: "OT_EUNSUPPORTED"}
BC_PERIODIC, BC_NEUMANN = 0, 1
PREC_MIXED, PREC_FP32, PREC_FP64 = 0, 1, 2


class OTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("ndim", c_int), ("n", c_int * 3), ("bc", c_int * 3), ("P", c_int), ("sigma", c_double),
                ("tau", c_double), ("axis_scale", c_double * 3), ("precision", c_int), ("check_every", c_int),
                ("lam_fp64", c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("residual", c_double), ("energy", c_double), ("mass_drift", c_double),
                ("elapsed_ms", c_double), ("dual_value", c_double), ("gap", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library() -> ctypes.CDLL:
    """Load libdynot.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdynot.so is not built; run __graft_entry__.build() "
                           "(or python -m paper_1501_04840_gb300._build)")
    lib = ctypes.CDLL(LIB_PATH)
    fp = POINTER(c_float)
    lib.ot_grid_rgb.argtypes = [POINTER(Grid), c_int, c_int, c_int]
    lib.ot_grid_rgb.restype = None
    lib.ot_grid_hue.argtypes = [POINTER(Grid), c_int, c_int]
    lib.ot_grid_hue.restype = None
    lib.ot_plan.argtypes = [POINTER(Grid), c_int, c_void_p, POINTER(c_void_p)]
    lib.ot_destroy.argtypes = [c_void_p]
    lib.ot_destroy.restype = None
    lib.ot_solve.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(Grid), c_int, c_double, c_void_p, POINTER(Stats)]
    lib.ot_solve_warm.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(Grid), c_int, c_double, c_void_p, c_void_p,
                                  c_int, c_double, c_double, POINTER(Stats), POINTER(c_int)]
    lib.ot_path.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_path_size.argtypes = [c_void_p]
    lib.ot_path_size.restype = c_size_t
    lib.ot_dual_size.argtypes = [c_void_p]
    lib.ot_dual_size.restype = c_size_t
    lib.ot_state_set.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_state_get.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_iterate.argtypes = [c_void_p, c_int, POINTER(Stats)]
    lib.ot_project.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_prox.argtypes = [c_int, c_int, c_double, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_prox_cardano.argtypes = [c_int, c_int, c_double, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_profile.argtypes = [c_void_p, c_int, POINTER(c_double), POINTER(c_char_p)]
    lib.ot_last_error.argtypes = []
    lib.ot_last_error.restype = c_char_p
    lib.ot_abi_version.restype = c_int
    lib.ot_batch_create.argtypes = [POINTER(Grid), c_int, c_void_p, POINTER(c_void_p)]
    lib.ot_batch_solve.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_void_p), c_int, c_double, c_int,
                                   POINTER(Stats)]
    lib.ot_batch_path.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.ot_batch_groups.argtypes = [c_void_p]
    lib.ot_batch_groups.restype = c_int
    lib.ot_batch_destroy.argtypes = [c_void_p]
    lib.ot_batch_destroy.restype = None
    for name in ("ot_plan", "ot_solve", "ot_solve_warm", "ot_path", "ot_state_set", "ot_state_get", "ot_iterate", "ot_project",
                 "ot_prox", "ot_prox_cardano", "ot_profile", "ot_batch_create", "ot_batch_solve", "ot_batch_path"):
        getattr(lib, name).restype = c_int
    del fp
    _lib = lib
    return lib


def _check(status: int, allow=()):
    if status != OT_OK and status not in allow:
        msg = load_library().ot_last_error().decode(errors="replace")
        raise OTError(status, msg)
    return status


def _ptr(a):
    """Pointer of a contiguous float32 numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be C-contiguous float32")
        return a.ctypes.data
    # torch tensor
    import torch  # noqa: WPS433 (optional dependency for device memory)
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float32")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def rgb_grid(n1: int, n2: int, P: int, **kw) -> Grid:
    g = Grid()
    load_library().ot_grid_rgb(ctypes.byref(g), n1, n2, P)
    for k, v in kw.items():
        _set(g, k, v)
    return g


def hue_grid(bins: int, P: int, **kw) -> Grid:
    g = Grid()
    load_library().ot_grid_hue(ctypes.byref(g), bins, P)
    for k, v in kw.items():
        _set(g, k, v)
    return g


def grid(n, bc, P, **kw) -> Grid:
    """General grid: n and bc are sequences of length ndim (bc: 'neumann' / 'periodic')."""
    g = rgb_grid(2, 2, P)
    g.ndim = len(n)
    for k in range(3):
        g.n[k] = n[k] if k < len(n) else 1
        b = bc[k] if k < len(bc) else "neumann"
        g.bc[k] = BC_PERIODIC if b in ("periodic", BC_PERIODIC) else BC_NEUMANN
    for k, v in kw.items():
        _set(g, k, v)
    return g


def _set(g, k, v):
    if k in ("n", "bc", "axis_scale"):
        arr = getattr(g, k)
        for i, x in enumerate(v):
            arr[i] = x
    else:
        setattr(g, k, v)


class Plan:
    """A solver plan: workspace for `batch` problems of one grid on one stream."""

    def __init__(self, g: Grid, batch: int = 1, stream: Optional[int] = None):
        self.lib = load_library()
        self.grid = g
        self.batch = batch
        h = c_void_p()
        _check(self.lib.ot_plan(ctypes.byref(g), batch, c_void_p(stream) if stream else None, ctypes.byref(h)))
        self.h = h
        nd = g.ndim
        n = [g.n[k] if k < nd else 1 for k in range(3)]
        self.n = n
        self.P = g.P
        self.S = n[0] * n[1] * n[2]
        self.N = self.P * self.S
        self.path_size = self.lib.ot_path_size(self.h)
        self.dual_size = self.lib.ot_dual_size(self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes of the compact path of one problem, in the ABI's layout
    def m_shape(self, k: int):
        nd = self.grid.ndim
        dims = list(self.n)
        if self.grid.bc[k] == BC_NEUMANN:
            dims[k] -= 1
        return (self.P, dims[2], dims[1], dims[0]) if nd == 3 else (
            (self.P, dims[1], dims[0]) if nd == 2 else (self.P, dims[0]))

    def f_shape(self):
        nd = self.grid.ndim
        return (self.P - 1, self.n[2], self.n[1], self.n[0]) if nd == 3 else (
            (self.P - 1, self.n[1], self.n[0]) if nd == 2 else (self.P - 1, self.n[0]))

    def cell_shape(self):
        return (self.P,) + self.f_shape()[1:]

    def solve(self, f0, f1, iters: int, tol: float = 0.0, init=None, check_every: int = 0) -> Stats:
        st = Stats()
        g = None
        if check_every:
            g = Grid.from_buffer_copy(self.grid)
            g.check_every = check_every
        s = self.lib.ot_solve(self.h, _ptr(f0), _ptr(f1), ctypes.byref(g) if g is not None else None, iters, tol,
                              _ptr(init), ctypes.byref(st))
        _check(s, allow=(OT_ENOTCONV,))
        st.converged = s == OT_OK
        return st

    def solve_warm(self, f0, f1, init, iters: int, tol: float = 0.0, dual_init: bool = True,
                   dual_support: float = 0.0, fallback_residual: float = 0.0, check_every: int = 0,
                   init_dual=None) -> Stats:
        """ot_solve_warm: start from the packed path `init` (and the packed dual `init_dual`, if given);
        st.used_cold tells whether it fell back to the cold start."""
        st = Stats()
        g = None
        if check_every:
            g = Grid.from_buffer_copy(self.grid)
            g.check_every = check_every
        used = c_int(0)
        s = self.lib.ot_solve_warm(self.h, _ptr(f0), _ptr(f1), ctypes.byref(g) if g is not None else None, iters,
                                   tol, _ptr(init), _ptr(init_dual), int(dual_init), dual_support, fallback_residual,
                                   ctypes.byref(st),
                                   ctypes.byref(used))
        _check(s, allow=(OT_ENOTCONV,))
        st.converged = s == OT_OK
        st.used_cold = bool(used.value)
        return st

    def path(self, out: str = "numpy", device=None):
        """Returns {'f': ..., 'm': [m_0, ..., m_{d-1}]} for all problems (leading batch axis)."""
        nd = self.grid.ndim
        B = self.batch

        def alloc(shape):
            if out == "numpy":
                return np.empty((B,) + tuple(shape), np.float32)
            import torch
            return torch.empty((B,) + tuple(shape), dtype=torch.float32, device=device or "cuda")

        f = alloc(self.f_shape())
        ms = [alloc(self.m_shape(k)) for k in range(nd)]
        ptrs = [_ptr(m) for m in ms] + [None] * (3 - nd)
        _check(self.lib.ot_path(self.h, _ptr(f), ptrs[0], ptrs[1], ptrs[2]))
        return {"f": f, "m": ms}

    def path_into(self, f, m0=None, m1=None, m2=None):
        """Copy the path into caller buffers (numpy or torch, host or device)."""
        _check(self.lib.ot_path(self.h, _ptr(f), _ptr(m0), _ptr(m1), _ptr(m2)))

    def state_set(self, f0, f1, x_packed, b_packed, bbar_packed=None):
        _check(self.lib.ot_state_set(self.h, _ptr(f0), _ptr(f1), _ptr(x_packed), _ptr(b_packed), _ptr(bbar_packed)))

    def state_get(self):
        x = np.empty(self.path_size, np.float32)
        b = np.empty(self.dual_size, np.float32)
        bb = np.empty(self.dual_size, np.float32)
        _check(self.lib.ot_state_get(self.h, _ptr(x), _ptr(b), _ptr(bb)))
        return x, b, bb

    def x_into(self, x_packed):
        """The primal x of the last check, packed, in solver units (mean density 1), into a caller buffer."""
        _check(self.lib.ot_state_get(self.h, _ptr(x_packed), None, None))

    def dual_into(self, b_packed):
        """The dual b of the last iteration, packed, into a caller buffer."""
        _check(self.lib.ot_state_get(self.h, None, _ptr(b_packed), None))

    def iterate(self, iters: int) -> Stats:
        st = Stats()
        _check(self.lib.ot_iterate(self.h, iters, ctypes.byref(st)))
        return st

    def project(self, f0, f1, a_packed, with_phi: bool = False):
        x = np.empty(self.path_size, np.float32)
        phi = np.empty(self.batch * self.N, np.float32) if with_phi else None
        _check(self.lib.ot_project(self.h, _ptr(f0), _ptr(f1), _ptr(a_packed), _ptr(x), _ptr(phi)))
        return (x, phi) if with_phi else x

    def profile(self, iters: int):
        ms = (c_double * 5)()
        names = c_char_p()
        _check(self.lib.ot_profile(self.h, iters, ms, ctypes.byref(names)))
        return dict(zip(names.value.decode().split(","), list(ms)))


class Batch:
    """Problems of mixed sizes solved together (C ABI ot_batch_*)."""

    def __init__(self, grids, stream: Optional[int] = None):
        self.lib = load_library()
        self.grids = list(grids)
        arr = (Grid * len(self.grids))(*self.grids)
        h = c_void_p()
        _check(self.lib.ot_batch_create(arr, len(self.grids), c_void_p(stream) if stream else None, ctypes.byref(h)))
        self.h = h
        self.shapes = []
        for g in self.grids:
            probe = Plan.__new__(Plan)
            probe.grid = g
            probe.n = [g.n[k] if k < g.ndim else 1 for k in range(3)]
            probe.P = g.P
            self.shapes.append(probe)

    @property
    def groups(self) -> int:
        return self.lib.ot_batch_groups(self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ot_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, f0s, f1s, iters: int, tol: float = 0.0, check_every: int = 0):
        n = len(self.grids)
        p0 = (c_void_p * n)(*[_ptr(a) for a in f0s])
        p1 = (c_void_p * n)(*[_ptr(a) for a in f1s])
        stats = (Stats * n)()
        s = self.lib.ot_batch_solve(self.h, p0, p1, iters, tol, check_every, stats)
        _check(s, allow=(OT_ENOTCONV,))
        out = list(stats)
        for st in out:
            st.converged = s == OT_OK
        return out

    def path(self, i: int):
        sh = self.shapes[i]
        f = np.empty(sh.f_shape(), np.float32)
        ms = [np.empty(sh.m_shape(k), np.float32) for k in range(sh.grid.ndim)]
        ptrs = [_ptr(m) for m in ms] + [None] * (3 - len(ms))
        _check(self.lib.ot_batch_path(self.h, i, _ptr(f), ptrs[0], ptrs[1], ptrs[2]))
        return {"f": f, "m": ms}


def prox(a_m, a_f, sigma: float, method: str = "newton"):
    """Per-cell prox of J on the device: a_m of shape (ncomp, count), a_f (count,); method 'newton' or 'cardano'."""
    lib = load_library()
    fn = lib.ot_prox if method == "newton" else lib.ot_prox_cardano
    a_m = np.ascontiguousarray(a_m, dtype=np.float32)
    a_f = np.ascontiguousarray(a_f, dtype=np.float32)
    ncomp, count = a_m.shape
    u = np.empty_like(a_m)
    v = np.empty_like(a_f)
    _check(fn(count, ncomp, sigma, _ptr(a_m), _ptr(a_f), _ptr(u), _ptr(v)))
    return u, v


def abi_version() -> int:
    return load_library().ot_abi_version()
