"""FP64 CPU oracle for the dynamic optimal-transport primal-dual iteration of
Fitschen, Laus & Steidl, "Dynamic Optimal Transport with Mixed Boundary
Conditions for Color Image Processing" (arXiv 1501.04840).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the package
entry file and the CPU-baseline leg of the benchmark may import this module.
The CUDA library never calls it and shares no code, table or constant with it.

Everything here is plain numpy in float64.  Library FFTs (scipy.fft.dct,
numpy.fft) serve as the transform steps of the Poisson solve; nothing is
blocked, fused or reordered beyond what the paper states.

Conventions (all arrays are numpy float64):

* ``Grid``: spatial axes k = 0..d-1 listed as (x, y, c) for RGB images or
  (hue,) for hue histograms; ``bc[k]`` is "neumann" (kappa = 1) or
  "periodic" (kappa = 0), section 2 "Discretization"; ``scale[k]`` is the
  factor of the difference matrices D_n / D_{n,per} (n in the paper, i.e. the
  unit cube of eq. (cont_model)); ``P`` is the number of time intervals p.
* Cell arrays (u, v, b, the Poisson unknown) have shape
  ``(P, n[d-1], ..., n[0])``: numpy axis 0 is the half-time index k - 1/2
  (k = 1..P), numpy axis ``d - k`` is spatial axis k.
* ``f`` has shape ``(P-1, n[d-1], ..., n[0])``: f[k-1] is f at time k/P,
  k = 1..P-1 (section 2, "Discretization").
* ``m`` is a list of d arrays.  m[k] has the cell shape except that spatial
  axis k holds n[k] - kappa faces.  Entry i along that axis is the paper's face
  j = i + kappa at position j/n: for Neumann the right face of cell i, for
  periodic the left face of cell i (face 0 sits at 0 == 1).

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.fft

NEUMANN = "neumann"
PERIODIC = "periodic"


@dataclass
class Grid:
    """Discrete grid of section 2: spatial sizes n, boundary kinds, scales, P."""

    n: Tuple[int, ...]
    bc: Tuple[str, ...]
    P: int
    scale: Optional[Tuple[float, ...]] = None

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.bc = tuple(self.bc)
        if len(self.n) != len(self.bc):
            raise ValueError("n and bc must have the same length")
        if self.scale is None:
            self.scale = tuple(float(v) for v in self.n)
        self.scale = tuple(float(v) for v in self.scale)
        if self.P < 2:
            raise ValueError("P >= 2 time intervals are required (f_b^- needs p >= 2)")
        for b in self.bc:
            if b not in (NEUMANN, PERIODIC):
                raise ValueError("bc must be 'neumann' or 'periodic'")

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def space_shape(self) -> Tuple[int, ...]:
        return tuple(reversed(self.n))

    @property
    def cell_shape(self) -> Tuple[int, ...]:
        return (self.P,) + self.space_shape

    @property
    def f_shape(self) -> Tuple[int, ...]:
        return (self.P - 1,) + self.space_shape

    def kappa(self, k: int) -> int:
        return 1 if self.bc[k] == NEUMANN else 0

    def m_shape(self, k: int) -> Tuple[int, ...]:
        s = list(self.cell_shape)
        s[self.ax(k)] = self.n[k] - self.kappa(k)
        return tuple(s)

    def ax(self, k: int) -> int:
        """numpy axis of spatial axis k in a cell/face/f array."""
        return self.d - k

    @property
    def ncells(self) -> int:
        return int(np.prod(self.cell_shape))

    @property
    def npix(self) -> int:
        return int(np.prod(self.n))


def rgb_grid(n1: int, n2: int, P: int, C: int = 3) -> Grid:
    """RGB image grid: Neumann in x and y, periodic colour (section 1, Remark 2)."""
    return Grid((n1, n2, C), (NEUMANN, NEUMANN, PERIODIC), P)


def hue_grid(nbins: int, P: int) -> Grid:
    """Hue-histogram grid: one periodic axis (section 5)."""
    return Grid((nbins,), (PERIODIC,), P)


# ---------------------------------------------------------------------------
# Interpolation S_M, S_F and their adjoints (section 2, definitions of S_M, S_F)
# ---------------------------------------------------------------------------

def _take(a: np.ndarray, axis: int, sl: slice) -> np.ndarray:
    idx = [slice(None)] * a.ndim
    idx[axis] = sl
    return a[tuple(idx)]


def _pad_zero(a: np.ndarray, axis: int, before: int, after: int) -> np.ndarray:
    pw = [(0, 0)] * a.ndim
    pw[axis] = (before, after)
    return np.pad(a, pw)


def S_M(g: Grid, m: Sequence[np.ndarray]) -> List[np.ndarray]:
    """u = S_M m: each cell takes the mean of its two faces along every axis.

    Neumann (S_M = I (x) S_n^T): the outermost faces j = 0, n are absent (zero).
    Periodic (S_M = I (x) S_{n,per}^T): cell i averages faces i and i+1 mod n.
    """
    out = []
    for k in range(g.d):
        ax = g.ax(k)
        mk = m[k]
        if g.bc[k] == NEUMANN:
            full = _pad_zero(mk, ax, 1, 1)             # faces j = 0..n
            left = _take(full, ax, slice(0, g.n[k]))
            right = _take(full, ax, slice(1, g.n[k] + 1))
        else:
            left = mk
            right = np.roll(mk, -1, axis=ax)
        out.append(0.5 * (left + right))
    return out


def S_M_T(g: Grid, u: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Adjoint S_M^T: each face takes the mean of its two neighbouring cells."""
    out = []
    for k in range(g.d):
        ax = g.ax(k)
        uk = u[k]
        if g.bc[k] == NEUMANN:
            out.append(0.5 * (_take(uk, ax, slice(0, g.n[k] - 1)) + _take(uk, ax, slice(1, g.n[k]))))
        else:
            out.append(0.5 * (np.roll(uk, 1, axis=ax) + uk))
    return out


def _time_stack(f0: np.ndarray, f: np.ndarray, f1: np.ndarray) -> np.ndarray:
    return np.concatenate([f0[None], f, f1[None]], axis=0)


def S_F(g: Grid, f: np.ndarray) -> np.ndarray:
    """S_F f = (S_p^T (x) I) f: half-time k-1/2 takes the mean of times k-1, k (ends zero)."""
    z = np.zeros(g.space_shape)
    F = _time_stack(z, f, z)
    return 0.5 * (F[:-1] + F[1:])


def f_b_plus(g: Grid, f0: np.ndarray, f1: np.ndarray) -> np.ndarray:
    """f_b^+ = 1/2 (f0, 0, ..., 0, f1) on the half-time cells (section 2)."""
    out = np.zeros(g.cell_shape)
    out[0] += 0.5 * f0
    out[-1] += 0.5 * f1
    return out


def f_b_minus(g: Grid, f0: np.ndarray, f1: np.ndarray) -> np.ndarray:
    """f_b^- = p (f0, 0, ..., 0, -f1) on the half-time cells (section 2)."""
    out = np.zeros(g.cell_shape)
    out[0] += g.P * f0
    out[-1] -= g.P * f1
    return out


def S_F_T(g: Grid, v: np.ndarray) -> np.ndarray:
    """Adjoint S_F^T = S_p (x) I: time k takes the mean of half-times k-1/2, k+1/2."""
    return 0.5 * (v[:-1] + v[1:])


def K(g: Grid, m: Sequence[np.ndarray], f: np.ndarray) -> Tuple[List[np.ndarray], np.ndarray]:
    """K = blockdiag(S_M, S_F) of Algorithm 1."""
    return S_M(g, m), S_F(g, f)


def K_T(g: Grid, bm: Sequence[np.ndarray], bf: np.ndarray) -> Tuple[List[np.ndarray], np.ndarray]:
    """K^T = blockdiag(S_M^T, S_F^T) of Algorithm 1, step 1."""
    return S_M_T(g, bm), S_F_T(g, bf)


# ---------------------------------------------------------------------------
# Divergence A = (D_M | D_F) and its adjoint (section 2, eq. (cont_d))
# ---------------------------------------------------------------------------

def D_M(g: Grid, m: Sequence[np.ndarray]) -> np.ndarray:
    """D_M m: forward difference of the faces of every cell, times the axis scale.

    Neumann: D_M = I (x) -D_n^T, i.e. n (m_right - m_left) with absent boundary
    faces.  Periodic: D_M = I (x) D_{n,per}^T, i.e. n (m_{i+1 mod n} - m_i).
    """
    out = np.zeros(g.cell_shape)
    for k in range(g.d):
        ax = g.ax(k)
        mk = m[k]
        if g.bc[k] == NEUMANN:
            full = _pad_zero(mk, ax, 1, 1)
            out += g.scale[k] * (_take(full, ax, slice(1, g.n[k] + 1)) - _take(full, ax, slice(0, g.n[k])))
        else:
            out += g.scale[k] * (np.roll(mk, -1, axis=ax) - mk)
    return out


def D_F(g: Grid, f: np.ndarray) -> np.ndarray:
    """D_F f = (-D_p^T (x) I) f: p (f_k - f_{k-1}) with the end values zero."""
    z = np.zeros(g.space_shape)
    F = _time_stack(z, f, z)
    return g.P * (F[1:] - F[:-1])


def A(g: Grid, m: Sequence[np.ndarray], f: np.ndarray) -> np.ndarray:
    """A (m, f) = D_M m + D_F f (section 2, eq. (cont_d))."""
    return D_M(g, m) + D_F(g, f)


def A_T(g: Grid, phi: np.ndarray) -> Tuple[List[np.ndarray], np.ndarray]:
    """A^T phi = (D_M^T phi, D_F^T phi).

    Neumann face i (paper face i+1): -n (phi_{i+1} - phi_i).
    Periodic face i (left face of cell i): n (phi_{i-1} - phi_i).
    f at time k: -p (phi_{k+1/2} - phi_{k-1/2}).
    """
    mt = []
    for k in range(g.d):
        ax = g.ax(k)
        if g.bc[k] == NEUMANN:
            mt.append(-g.scale[k] * (_take(phi, ax, slice(1, g.n[k])) - _take(phi, ax, slice(0, g.n[k] - 1))))
        else:
            mt.append(g.scale[k] * (np.roll(phi, 1, axis=ax) - phi))
    ft = -g.P * (phi[1:] - phi[:-1])
    return mt, ft


# ---------------------------------------------------------------------------
# Poisson solve (A A^T)^dagger (section 3, step 1; Remark 2)
# ---------------------------------------------------------------------------

def eigenvalues(g: Grid) -> np.ndarray:
    """Eigenvalues of A A^T on the cell grid, in transform order.

    A A^T = sum over spatial axes of s_k^2 Delta_k (x) I + p^2 Delta_p (x) I, with
    Delta_{n,per} = (1/n) conj(F_n) diag(4 sin^2(j pi/n)) F_n and
    Delta_p = C_p^T diag(4 sin^2(j pi/(2p))) C_p (section 3); a Neumann spatial
    axis has the same form as the time axis.
    """
    lam = np.zeros(g.cell_shape)
    jt = np.arange(g.P)
    sh = [1] * (g.d + 1)
    sh[0] = g.P
    lam = lam + (g.P ** 2 * 4.0 * np.sin(jt * np.pi / (2 * g.P)) ** 2).reshape(sh)
    for k in range(g.d):
        j = np.arange(g.n[k])
        if g.bc[k] == NEUMANN:
            q = 4.0 * np.sin(j * np.pi / (2 * g.n[k])) ** 2
        else:
            q = 4.0 * np.sin(j * np.pi / g.n[k]) ** 2
        sh = [1] * (g.d + 1)
        sh[g.ax(k)] = g.n[k]
        lam = lam + (g.scale[k] ** 2 * q).reshape(sh)
    return lam


def poisson_pinv(g: Grid, r: np.ndarray) -> np.ndarray:
    """phi = (A A^T)^dagger r by the spectral decomposition of section 3.

    Forward: orthonormal DCT-II C_p along time and every Neumann axis, DFT F_n
    along every periodic axis.  Divide by the eigenvalue; the zero eigenvalue is
    mapped to zero (pseudo-inverse).  Inverse transforms back.
    """
    lam = eigenvalues(g)
    h = scipy.fft.dct(r, type=2, norm="ortho", axis=0)
    for k in range(g.d):
        ax = g.ax(k)
        if g.bc[k] == NEUMANN:
            h = scipy.fft.dct(h, type=2, norm="ortho", axis=ax)
        else:
            h = np.fft.fft(h, axis=ax)
    inv = np.zeros_like(lam)
    nz = lam > 0
    inv[nz] = 1.0 / lam[nz]
    h = h * inv
    for k in range(g.d):
        ax = g.ax(k)
        if g.bc[k] == NEUMANN:
            h = scipy.fft.idct(h, type=2, norm="ortho", axis=ax)
        else:
            h = np.fft.ifft(h, axis=ax)
    h = scipy.fft.idct(h, type=2, norm="ortho", axis=0)
    return np.real(h)


def project(g: Grid, am: Sequence[np.ndarray], af: np.ndarray, f0: np.ndarray, f1: np.ndarray):
    """Pi_{C_d}(a) = a - A^T (A A^T)^dagger (A a - f_b^-)  (section 3, step 1).

    Returns (m, f, phi) where phi = (A A^T)^dagger (A a - f_b^-).
    """
    r = A(g, am, af) - f_b_minus(g, f0, f1)
    phi = poisson_pinv(g, r)
    mt, ft = A_T(g, phi)
    m = [am[k] - mt[k] for k in range(g.d)]
    f = af - ft
    return m, f, phi


# ---------------------------------------------------------------------------
# Proximal map of the kinetic energy (section 3, step 2)
# ---------------------------------------------------------------------------

def prox_J(am: Sequence[np.ndarray], af: np.ndarray, sigma: float,
           tol: float = 1e-15, max_iter: int = 500):
    """Per-cell argmin_{u,v} |u|^2/(2v) + sigma/2 |u - a_m|^2 + sigma/2 (v - a_f)^2.

    Zero gradient gives u = sigma v a_m / (1 + sigma v), with v the root of the
    cubic g(v) = 2 (1 + sigma v)^2 (v - a_f) - sigma |a_m|^2 (section 3, step 2).
    g has a positive root iff g(0) < 0, i.e. a_f + sigma |a_m|^2 / 2 > 0; otherwise
    the minimiser is (u, v) = (0, 0), the only point of the domain of J with
    v <= 0 where J is finite.  Newton's method ("few Newton steps") starts at
    v0 = a_f + sigma |a_m|^2 / 2, where g(v0) = sigma |a_m|^2 ((1+sigma v0)^2 - 1) >= 0,
    and g is increasing and convex on [root, v0], so the iterates decrease
    monotonically to the root.  Iterates until |dv| <= tol * v.
    """
    shape = np.shape(af)
    am = [np.asarray(a, dtype=np.float64).reshape(-1) for a in am]
    af = np.asarray(af, dtype=np.float64).reshape(-1)
    s2 = np.zeros_like(af)
    for a in am:
        s2 = s2 + a * a
    pos = af + 0.5 * sigma * s2 > 0
    v = np.where(pos, af + 0.5 * sigma * s2, 0.0)
    idx = np.flatnonzero(pos)
    for _ in range(max_iter):
        if idx.size == 0:
            break
        va = v[idx]
        afa = af[idx]
        w = 1.0 + sigma * va
        gval = 2.0 * w * w * (va - afa) - sigma * s2[idx]
        dg = 4.0 * sigma * w * (va - afa) + 2.0 * w * w
        step = gval / dg
        vn = va - step
        v[idx] = vn
        idx = idx[np.abs(step) > tol * np.abs(vn)]
    u = [np.where(pos, sigma * v * a / (1.0 + sigma * v), 0.0).reshape(shape) for a in am]
    v = np.where(pos, v, 0.0).reshape(shape)
    return u, v


def J_energy(u: Sequence[np.ndarray], v: np.ndarray) -> np.ndarray:
    """Per-cell J(u, v) of eq. (cont_model): |u|^2/(2v) for v > 0, 0 at (0,0), inf otherwise."""
    s2 = np.zeros_like(v)
    for a in u:
        s2 = s2 + a * a
    out = np.full(v.shape, np.inf)
    pos = v > 0
    out[pos] = s2[pos] / (2.0 * v[pos])
    out[(v == 0) & (s2 == 0)] = 0.0
    return out


# ---------------------------------------------------------------------------
# Algorithm 1 (PDHG, theta = 1)
# ---------------------------------------------------------------------------

@dataclass
class State:
    """Primal x = (m, f), scaled dual b = (b_m, b_f) and its extrapolation bbar."""

    m: List[np.ndarray]
    f: np.ndarray
    bm: List[np.ndarray]
    bf: np.ndarray
    bbm: List[np.ndarray]
    bbf: np.ndarray

    @staticmethod
    def zeros(g: Grid) -> "State":
        """Initialisation of Algorithm 1: every variable zero."""
        return State([np.zeros(g.m_shape(k)) for k in range(g.d)], np.zeros(g.f_shape),
                     [np.zeros(g.cell_shape) for _ in range(g.d)], np.zeros(g.cell_shape),
                     [np.zeros(g.cell_shape) for _ in range(g.d)], np.zeros(g.cell_shape))

    def copy(self) -> "State":
        return State([a.copy() for a in self.m], self.f.copy(), [a.copy() for a in self.bm],
                     self.bf.copy(), [a.copy() for a in self.bbm], self.bbf.copy())


@dataclass
class StepInfo:
    residual: float          # ||b^{r+1} - b^r|| / ||K x^{r+1} + (0, f_b^+)||
    primal_change: float     # ||x^{r+1} - x^r|| / ||x^{r+1}||
    continuity: float        # ||A x^{r+1} - f_b^-|| / ||f_b^-||
    energy: float            # (1/#cells) sum J(u^{r+1}, v^{r+1})
    dual: Optional[float] = None   # dual_value at p = sigma b^{r+1} (when the step is given x0)
    u: List[np.ndarray] = field(repr=False, default=None)
    v: np.ndarray = field(repr=False, default=None)


def _norm2(arrs) -> float:
    return float(np.sqrt(sum(float(np.sum(a * a)) for a in arrs)))


def min_norm_path(g: Grid, f0: np.ndarray, f1: np.ndarray) -> Tuple[List[np.ndarray], np.ndarray]:
    """x0 = Pi_{C_d}(0) = A^T (A A^T)^+ f_b^-: the path of least norm that meets the continuity
    constraint (the projection of section 3 applied to a = 0)."""
    zm = [np.zeros(g.m_shape(k)) for k in range(g.d)]
    m, f, _ = project(g, zm, np.zeros(g.f_shape), f0, f1)
    return m, f


def dual_value(g: Grid, bm: Sequence[np.ndarray], bf: np.ndarray, x0, f0: np.ndarray, f1: np.ndarray,
               sigma: float) -> float:
    """Dual objective of the discrete problem at p = sigma b, per cell (no counterpart in the paper).

    The problem is min over x in C_d of ||J(K x + (0, f_b^+))||_1.  Its Lagrangian dual function at p is
    -J*(p) + <p_f, f_b^+> + inf_{x in C_d} <K^T p, x>.  J is the support function of
    {(a, b): b + |a|^2 / 2 <= 0}, so J* = 0 on that set; step 2 of Algorithm 1 puts sigma b^{r+1} in the
    subdifferential of J at (u, v), hence in it.  The infimum over C_d = x0 + ker A equals <K^T p, x0>
    when K^T p lies in the range of A^T (the dual constraint), and this value is taken:
        D = sigma (<b_m, S_M m0> + <b_f, S_F f0 + f_b^+>) / #cells,  (m0, f0) = min_norm_path.
    At a saddle point the primal energy (1/#cells) sum J(u, v) equals D; the difference is the
    primal-dual gap."""
    sm, sf = K(g, x0[0], x0[1])
    fbp = f_b_plus(g, f0, f1)
    tot = sum(float(np.sum(bm[k] * sm[k])) for k in range(g.d)) + float(np.sum(bf * (sf + fbp)))
    return sigma * tot / g.ncells


def pdhg_step(g: Grid, st: State, f0: np.ndarray, f1: np.ndarray, sigma: float, tau: float,
              theta: float = 1.0, x0=None) -> Tuple[State, StepInfo]:
    """One iteration of Algorithm 1 (steps 1-4), in the paper's order.  With x0 = min_norm_path the
    step also reports the dual value of its dual iterate."""
    # step 1: x^{r+1} = Pi_{C_d}(x^r - tau sigma K^T bbar^r)
    km, kf = K_T(g, st.bbm, st.bbf)
    am = [st.m[k] - tau * sigma * km[k] for k in range(g.d)]
    af = st.f - tau * sigma * kf
    m, f, _ = project(g, am, af, f0, f1)
    # step 2: (u, v) = prox_{J/sigma}(K x^{r+1} + (0, f_b^+) + b^r)
    sm, sf = K(g, m, f)
    fbp = f_b_plus(g, f0, f1)
    a_m = [sm[k] + st.bm[k] for k in range(g.d)]
    a_f = sf + fbp + st.bf
    u, v = prox_J(a_m, a_f, sigma)
    # step 3: b^{r+1} = b^r + K x^{r+1} + (0, f_b^+) - (u, v)
    bm = [a_m[k] - u[k] for k in range(g.d)]
    bf = a_f - v
    # step 4: bbar^{r+1} = b^{r+1} + theta (b^{r+1} - b^r)
    bbm = [bm[k] + theta * (bm[k] - st.bm[k]) for k in range(g.d)]
    bbf = bf + theta * (bf - st.bf)
    new = State(m, f, bm, bf, bbm, bbf)
    db = [bm[k] - st.bm[k] for k in range(g.d)] + [bf - st.bf]
    kx = list(sm) + [sf + fbp]
    dx = [m[k] - st.m[k] for k in range(g.d)] + [f - st.f]
    fbm = f_b_minus(g, f0, f1)
    info = StepInfo(
        residual=_norm2(db) / max(_norm2(kx), 1e-300),
        primal_change=_norm2(dx) / max(_norm2(list(m) + [f]), 1e-300),
        continuity=_norm2([A(g, m, f) - fbm]) / max(_norm2([fbm]), 1e-300),
        energy=float(np.sum(J_energy(u, v))) / g.ncells,
        dual=None if x0 is None else dual_value(g, bm, bf, x0, f0, f1, sigma),
        u=u, v=v)
    return new, info


def warm_state(g: Grid, m: Sequence[np.ndarray], f: np.ndarray, f0: np.ndarray, f1: np.ndarray,
               sigma: float, dual: bool = True, vmin: float = 1e-3, wmax: Optional[float] = None,
               support: float = 0.0) -> State:
    """Initial state of Algorithm 1 from a given path x0 = (m, f) (no counterpart in the paper).

    Without ``dual`` the dual starts at zero as in Algorithm 1.  With it,
    b = bbar = grad J(y) / sigma at y = K x0 + (0, f_b^+): step 2 has the
    optimality condition 0 = grad J(y) + sigma (y - K x - (0, f_b^+) - b), and
    step 3 leaves b unchanged exactly when y = K x + (0, f_b^+).  grad J(u, v)
    = (w, -|w|^2 / 2) with the velocity w = u / v, for J = |u|^2 / (2 v); v is
    clamped below by vmin and |w| above by wmax, by default the diameter of the
    domain (each axis spans n / scale, half of that when periodic): an optimal
    path moves no mass faster than that per unit time.  Cells whose density is
    below ``support`` keep b = 0: where the density vanishes, the dual of an
    optimal path may be any point of the subdifferential of J at 0.
    """
    st = State.zeros(g)
    st.m = [np.asarray(a, float).copy() for a in m]
    st.f = np.asarray(f, float).copy()
    if dual:
        if wmax is None:
            wmax = float(np.sqrt(sum((g.n[k] / g.scale[k] * (0.5 if g.bc[k] == PERIODIC else 1.0)) ** 2
                                     for k in range(g.d))))
        sm, sf = K(g, st.m, st.f)
        vraw = sf + f_b_plus(g, f0, f1)
        v = np.maximum(vraw, vmin)
        on = (vraw >= support).astype(float)
        w = [on * a / v for a in sm]
        speed = np.sqrt(sum(a * a for a in w))
        lim = np.where(speed > wmax, wmax / np.maximum(speed, 1e-300), 1.0)
        w = [a * lim for a in w]
        st.bm = [a / sigma for a in w]
        st.bf = -sum(a * a for a in w) / (2.0 * sigma)
        st.bbm = [a.copy() for a in st.bm]
        st.bbf = st.bf.copy()
    return st


def normalise_pair(g: Grid, f0: np.ndarray, f1: np.ndarray, rel_tol: float = 1e-6):
    """Mass rescaling of section 4 (||f0||_1 = ||f1||_1) to mean density 1.

    Both densities are scaled so that their sum over the spatial cells equals
    the number of spatial cells.  Returns (g0, g1, out_scale) where the solver's
    path, multiplied by out_scale, is in the caller's units.
    """
    f0 = np.asarray(f0, dtype=np.float64)
    f1 = np.asarray(f1, dtype=np.float64)
    if f0.shape != g.space_shape or f1.shape != g.space_shape:
        raise ValueError("f0/f1 must have shape %s" % (g.space_shape,))
    if (f0 < 0).any() or (f1 < 0).any() or not np.isfinite(f0).all() or not np.isfinite(f1).all():
        raise ValueError("densities must be finite and non-negative")
    M0, M1 = float(f0.sum()), float(f1.sum())
    if M0 <= 0 or M1 <= 0 or abs(M0 - M1) > rel_tol * max(M0, M1):
        raise ValueError("masses differ: %r vs %r" % (M0, M1))
    T = float(g.npix)
    return f0 * (T / M0), f1 * (T / M1), 0.5 * (M0 + M1) / T


def solve(g: Grid, f0: np.ndarray, f1: np.ndarray, iters: int, sigma: float, tau: float,
          state: Optional[State] = None, normalise: bool = True, tol: float = 0.0,
          check_every: int = 1, callback=None, with_dual: bool = False):
    """Run Algorithm 1 for ``iters`` iterations (or until residual <= tol).

    With ``normalise`` the pair is rescaled by :func:`normalise_pair` first and
    the returned path is scaled back.  Returns (state, infos, scale) where the
    state is in solver units and ``scale`` maps its m, f and energy back.
    ``with_dual`` adds the dual value of every iterate (info.dual).
    """
    if normalise:
        g0, g1, scale = normalise_pair(g, f0, f1)
    else:
        g0, g1, scale = np.asarray(f0, float), np.asarray(f1, float), 1.0
    st = State.zeros(g) if state is None else state.copy()
    x0 = min_norm_path(g, g0, g1) if with_dual else None
    infos = []
    for r in range(iters):
        st, info = pdhg_step(g, st, g0, g1, sigma, tau, x0=x0)
        info.u = info.v = None
        infos.append(info)
        if callback is not None:
            callback(r, st, info)
        if tol > 0 and check_every > 0 and (r + 1) % check_every == 0 and info.residual <= tol:
            break
    return st, infos, scale
