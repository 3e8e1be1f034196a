"""Learned warm start for Algorithm 1.

A 3D U-Net over (t, y, x) maps the boundary densities (f0, f1) of an RGB
pair to an initial path x0 = (m_x, m_y, m_c, f) on the P-step staggered grid
and an initial dual b0 (the scaled dual of Algorithm 1 at the cells);
ot_solve_warm then starts Algorithm 1 from them (its first step projects
x0 - tau sigma K^T b0 onto the continuity constraint).  The network predicts f
as a deviation from the linear interpolation (1 - t) f0 + t f1.  The plain
cold start remains the fallback when the warm start's first residual is worse
than a cold start's.

Every numerical step runs in libdynot.so (convolutions on the tensor cores with
bf16 operands and fp32 accumulation, pooling, losses, AdamW, the solver);
torch provides device memory and the stream.  The paper has no network: this
is an addition on top of its method.

Densities are handled in solver units (mean density 1): ``to_solver_units``
rescales a pair on the host before upload, so the network's inputs and targets
and the solver's path share one scale.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import time
from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch

from . import nn as K
from .binding import Plan, rgb_grid
from .synth import rgb_pair

WIDTHS = (16, 32, 48, 64)
# weights trained by `python -m paper_1501_04840_gb300.warmstart` (2000 pairs at 128x128x3, P = 32, 6000 steps)
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_rgb128x128x3x32.npz")
CIN = 16    # input channels: f0 (3), f1 (3), interpolation (3), half time (1), zero padding
COUT = 32   # output channels: 12 path channels (m_x, m_y, m_c, f deviation; 3 colours each),
CV = 24     # then 12 dual channels (b_mx, b_my, b_mc, b_f), then 8 unused
DUAL0 = 12


@contextlib.contextmanager
def side_stream():
    """Run on a non-default torch stream: the solver plans made here share it (their own streams are
    non-blocking and would not order against the legacy default stream)."""
    cur = torch.cuda.current_stream()
    if cur.cuda_stream != 0:
        yield cur
        return
    s = torch.cuda.Stream()
    s.wait_stream(cur)
    with torch.cuda.stream(s):
        yield s
    cur.wait_stream(s)


def to_solver_units(f0: np.ndarray, f1: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Rescale both densities to mean 1 over pixels and channels (float32)."""
    S = f0.size
    return ((f0.astype(np.float64) * (S / f0.astype(np.float64).sum())).astype(np.float32),
            (f1.astype(np.float64) * (S / f1.astype(np.float64).sum())).astype(np.float32))


def conv_specs(widths=WIDTHS, cin: int = CIN, cout: int = COUT) -> List[Tuple[str, int, int]]:
    """(name, input channels, output channels) of every convolution, forward order.

    Encoder level l: e{l}a, e{l}b; decoder level l (deepest first) takes the
    upsampled deeper output concatenated with the level's skip: d{l}a, d{l}b;
    then a linear head.
    """
    L = len(widths)
    out, c = [], cin
    for l in range(L):
        out.append(("e%da" % l, c, widths[l]))
        out.append(("e%db" % l, widths[l], widths[l]))
        c = widths[l]
    for l in range(L - 2, -1, -1):
        out.append(("d%da" % l, widths[l + 1] + widths[l], widths[l]))
        out.append(("d%db" % l, widths[l], widths[l]))
    out.append(("head", widths[0], cout))
    return out


class _Buffers:
    """Activations (and, for training, their gradients) for one batch shape."""

    def __init__(self, widths, N, P, Y, X, train: bool, device):
        L = len(widths)
        if Y % (1 << (L - 1)) or X % (1 << (L - 1)):
            raise ValueError("Y and X must be divisible by %d" % (1 << (L - 1)))
        self.vols = [(N, P, Y >> l, X >> l) for l in range(L)]
        bf = dict(dtype=torch.bfloat16, device=device)

        def act(l, c):
            return torch.empty(self.vols[l] + (c,), **bf)

        self.inp = act(0, CIN)
        self.ea = [act(l, widths[l]) for l in range(L)]
        self.cat = [act(l, widths[l + 1] + widths[l]) for l in range(L - 1)]
        self.bott = act(L - 1, widths[L - 1])
        self.pl = [act(l + 1, widths[l]) for l in range(L - 1)]
        self.da = [act(l, widths[l]) for l in range(L - 1)]
        self.db = [act(l, widths[l]) for l in range(L - 1)]
        self.out = torch.empty(self.vols[0] + (COUT,), dtype=torch.float32, device=device)
        self.train = train
        if train:
            self.g_out = act(0, COUT)
            self.g_db = [act(l, widths[l]) for l in range(L - 1)]
            self.g_da = [act(l, widths[l]) for l in range(L - 1)]
            self.g_cat = [act(l, widths[l + 1] + widths[l]) for l in range(L - 1)]
            self.g_bott = act(L - 1, widths[L - 1])
            self.g_ea = [act(l, widths[l]) for l in range(L)]
            self.g_pl = [act(l + 1, widths[l]) for l in range(L - 1)]
            self.tmp = [act(l, widths[l]) for l in range(L - 1)]
            self.loss = torch.zeros(1, dtype=torch.float32, device=device)


class UNet:
    """The warm-start network: parameters, forward, backward and AdamW."""

    def __init__(self, widths=WIDTHS, seed: int = 0, device: str = "cuda", params: Optional[np.ndarray] = None):
        self.widths = tuple(widths)
        self.L = len(self.widths)
        self.device = device
        self.specs = conv_specs(self.widths)
        self.off: Dict[str, Tuple[int, int, int, int]] = {}
        pos = 0
        for name, ci, co in self.specs:
            nw = co * 27 * ci
            wo = pos
            pos += (nw + 63) // 64 * 64
            bo = pos
            pos += (co + 63) // 64 * 64
            self.off[name] = (wo, nw, bo, co)
        self.size = pos
        if params is None:
            params = self.init_params(seed)
        f32 = dict(dtype=torch.float32, device=device)
        self.p32 = torch.from_numpy(np.ascontiguousarray(params, np.float32)).to(device)
        self.g32 = torch.zeros(self.size, **f32)
        self.m = torch.zeros(self.size, **f32)
        self.v = torch.zeros(self.size, **f32)
        self.pb = torch.empty(self.size, dtype=torch.bfloat16, device=device)
        self.wr = torch.empty(self.size, dtype=torch.bfloat16, device=device)
        self.step = 0
        self._bufs: Dict[tuple, _Buffers] = {}
        K.to_bf16(self.p32, self.pb)
        self._rotated = False

    @property
    def n_params(self) -> int:
        return sum(co * 27 * ci + co for _, ci, co in self.specs)

    def init_params(self, seed: int) -> np.ndarray:
        """He-normal weights for the ReLU layers, a small head (the first prediction is the interpolation)."""
        rng = np.random.default_rng(seed)
        p = np.zeros(self.size, np.float32)
        for name, ci, co in self.specs:
            wo, nw, _, _ = self.off[name]
            std = math.sqrt(2.0 / (27 * ci)) if name != "head" else 1e-3
            p[wo:wo + nw] = rng.standard_normal(nw) * std
        return p

    def params_numpy(self) -> Dict[str, Tuple[np.ndarray, np.ndarray]]:
        """{name: (w [cout][27][cin], b [cout])} of the fp32 master weights."""
        p = self.p32.cpu().numpy()
        out = {}
        for name, ci, co in self.specs:
            wo, nw, bo, _ = self.off[name]
            out[name] = (p[wo:wo + nw].reshape(co, 27, ci).copy(), p[bo:bo + co].copy())
        return out

    def grads_numpy(self) -> Dict[str, Tuple[np.ndarray, np.ndarray]]:
        g = self.g32.cpu().numpy()
        out = {}
        for name, ci, co in self.specs:
            wo, nw, bo, _ = self.off[name]
            out[name] = (g[wo:wo + nw].reshape(co, 27, ci).copy(), g[bo:bo + co].copy())
        return out

    # parameter views
    def _w(self, name):
        wo, nw, _, _ = self.off[name]
        return self.pb[wo:wo + nw]

    def _wr(self, name):
        wo, nw, _, _ = self.off[name]
        return self.wr[wo:wo + nw]

    def _b(self, name):
        _, _, bo, co = self.off[name]
        return self.p32[bo:bo + co]

    def _gw(self, name):
        wo, nw, _, _ = self.off[name]
        return self.g32[wo:wo + nw]

    def _gb(self, name):
        _, _, bo, co = self.off[name]
        return self.g32[bo:bo + co]

    def buffers(self, N, P, Y, X, train: bool) -> _Buffers:
        key = (N, P, Y, X, train)
        if key not in self._bufs:
            self._bufs[key] = _Buffers(self.widths, N, P, Y, X, train, self.device)
        return self._bufs[key]

    def _skip(self, B: _Buffers, l: int) -> K.Slice:
        if l == self.L - 1:
            return K.whole(B.bott)
        return K.Slice(B.cat[l], self.widths[l + 1], self.widths[l])

    # ---- forward
    def forward(self, B: _Buffers, stream=None):
        W, w = self.widths, K.whole
        x = w(B.inp)
        for l in range(self.L):
            K.conv3d(B.vols[l], x, self._w("e%da" % l), self._b("e%da" % l), w(B.ea[l]), True, stream=stream)
            s = self._skip(B, l)
            K.conv3d(B.vols[l], w(B.ea[l]), self._w("e%db" % l), self._b("e%db" % l), s, True, stream=stream)
            if l < self.L - 1:
                K.pool(B.vols[l + 1], s, w(B.pl[l]), stream=stream)
                x = w(B.pl[l])
        h = w(B.bott)
        for l in range(self.L - 2, -1, -1):
            K.upsample(B.vols[l + 1], h, K.Slice(B.cat[l], 0, W[l + 1]), stream=stream)
            K.conv3d(B.vols[l], w(B.cat[l]), self._w("d%da" % l), self._b("d%da" % l), w(B.da[l]), True,
                     stream=stream)
            K.conv3d(B.vols[l], w(B.da[l]), self._w("d%db" % l), self._b("d%db" % l), w(B.db[l]), True,
                     stream=stream)
            h = w(B.db[l])
        K.conv3d(B.vols[0], h, self._w("head"), self._b("head"), w(B.out), False, out_f32=True, stream=stream)
        return B.out

    # ---- backward (gradients accumulate into g32, which the caller zeroes)
    def _back(self, name, vol, xin, y, gy, gx, stream):
        if y is not None:
            K.relu_grad(gy, y, stream=stream)
        K.conv3d_wgrad(vol, xin, gy, self._gw(name), self._gb(name), stream=stream)
        if gx is not None:
            K.conv3d(vol, gy, self._wr(name), None, gx, False, stream=stream)

    def rotate(self, stream=None):
        for name, ci, co in self.specs:
            K.rotate_weights(ci, co, self._w(name), self._wr(name), stream=stream)

    def backward(self, B: _Buffers, target: torch.Tensor, stream=None):
        """MSE of the CV output channels against the bf16 target [N][P][Y][X][CV]; loss accumulates in B.loss."""
        W, w = self.widths, K.whole
        self.rotate(stream)
        K.mse(B.out, CV, target, B.g_out, B.loss, stream=stream)
        self._back("head", B.vols[0], w(B.db[0]), None, w(B.g_out), w(B.g_db[0]), stream)
        for l in range(self.L - 1):
            self._back("d%db" % l, B.vols[l], w(B.da[l]), w(B.db[l]), w(B.g_db[l]), w(B.g_da[l]), stream)
            self._back("d%da" % l, B.vols[l], w(B.cat[l]), w(B.da[l]), w(B.g_da[l]), w(B.g_cat[l]), stream)
            deeper = w(B.g_db[l + 1]) if l + 1 < self.L - 1 else w(B.g_bott)
            K.upsample(B.vols[l + 1], K.Slice(B.g_cat[l], 0, W[l + 1]), deeper, backward=True, stream=stream)
        gs = w(B.g_bott)
        for l in range(self.L - 1, -1, -1):
            if l < self.L - 1:
                K.pool(B.vols[l + 1], w(B.g_pl[l]), w(B.tmp[l]), backward=True, stream=stream)
                gs = K.Slice(B.g_cat[l], W[l + 1], W[l])
                K.add_slice(w(B.tmp[l]), gs, stream=stream)
            self._back("e%db" % l, B.vols[l], w(B.ea[l]), self._skip(B, l), gs, w(B.g_ea[l]), stream)
            xin = w(B.inp) if l == 0 else w(B.pl[l - 1])
            self._back("e%da" % l, B.vols[l], xin, w(B.ea[l]), w(B.g_ea[l]), w(B.g_pl[l - 1]) if l > 0 else None,
                       stream)

    def adamw(self, lr, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4, stream=None):
        self.step += 1
        K.adamw(self.p32, self.g32, self.m, self.v, self.pb, lr, b1, b2, eps, wd, self.step, stream=stream)

    # ---- inference: the packed initial path (solver units) and packed dual of N pairs
    def predict(self, f0: torch.Tensor, f1: torch.Tensor, P: int, init: torch.Tensor, dual=None, stream=None):
        N, _, Y, X = f0.shape
        B = self.buffers(N, P, Y, X, False)
        K.make_input(N, P, Y, X, f0, f1, B.inp, stream=stream)
        self.forward(B, stream)
        K.path_channels(N, Y, X, P, False, init, B.out, f0=f0, f1=f1, stream=stream)
        if dual is not None:
            K.dual_channels(N, Y, X, P, False, dual, B.out, DUAL0, stream=stream)
        return init

    def save(self, path: str, **meta):
        np.savez(path, params=self.p32.cpu().numpy(), widths=np.array(self.widths),
                 meta=json.dumps(meta))

    @staticmethod
    def load(path: str, device: str = "cuda") -> Tuple["UNet", dict]:
        z = np.load(path)
        net = UNet(tuple(int(w) for w in z["widths"]), device=device, params=z["params"])
        return net, json.loads(str(z["meta"]))


# ---------------------------------------------------------------------------
# data: solver-generated (f0, f1) -> path pairs
# ---------------------------------------------------------------------------

@dataclass
class PairSet:
    f0: torch.Tensor       # [n][3][Y][X] solver units (device)
    f1: torch.Tensor
    target: Optional[torch.Tensor]   # [n][P][Y][X][CV] bf16 path and dual channels (device) or None
    seeds: List[int]
    iterations: List[int]


def make_pairs(seeds, side: int, nblobs: int, device="cuda") -> Tuple[torch.Tensor, torch.Tensor]:
    f0s, f1s = [], []
    for s in seeds:
        a, b = rgb_pair(side, side, nblobs, s)
        a, b = to_solver_units(a, b)
        f0s.append(a)
        f1s.append(b)
    return (torch.from_numpy(np.stack(f0s)).to(device), torch.from_numpy(np.stack(f1s)).to(device))


def _solve_targets(seeds, side: int, P: int, nblobs: int, batch: int = 16, tol: float = 1e-5,
                   max_iters: int = 6000, device="cuda", log=None) -> PairSet:
    """Solve every pair with the cold-started GPU solver; keep its path and dual as CV bf16 channels."""
    f0, f1 = make_pairs(seeds, side, nblobs, device)
    n = len(seeds)
    target = torch.empty((n, P, side, side, CV), dtype=torch.bfloat16, device=device)
    tmp = torch.empty((min(batch, n), P, side, side, CV), dtype=torch.float32, device=device)
    iters = []
    stream = torch.cuda.current_stream()
    plans, xbuf = {}, {}
    for i0 in range(0, n, batch):
        nb = min(batch, n - i0)
        if nb not in plans:
            plans[nb] = Plan(rgb_grid(side, side, P), batch=nb, stream=stream.cuda_stream)
            xbuf[nb] = (torch.empty(plans[nb].path_size, dtype=torch.float32, device=device),
                        torch.empty(plans[nb].dual_size, dtype=torch.float32, device=device))
        plan, (x, b) = plans[nb], xbuf[nb]
        st = plan.solve(f0[i0:i0 + nb], f1[i0:i0 + nb], max_iters, tol)
        plan.x_into(x)
        plan.dual_into(b)
        t = tmp[:nb]
        K.path_channels(nb, side, side, P, True, x, t, f0=f0[i0:i0 + nb], f1=f1[i0:i0 + nb], stream=stream)
        K.dual_channels(nb, side, side, P, True, b, t, DUAL0, stream=stream)
        K.to_bf16(t, target[i0:i0 + nb], stream=stream)
        iters += [st.iterations] * nb
        if log:
            log("targets %d/%d: %d iterations, residual %.2e" % (i0 + nb, n, st.iterations, st.residual))
    for p in plans.values():
        p.close()
    torch.cuda.synchronize()
    return PairSet(f0, f1, target, list(seeds), iters)


# ---------------------------------------------------------------------------
# training and evaluation
# ---------------------------------------------------------------------------

def _train(net: UNet, data: PairSet, P: int, steps: int, batch: int = 4, lr: float = 2e-3, lr_min: float = 2e-5,
          seed: int = 0, log=None, log_every: int = 50) -> List[float]:
    """AdamW with cosine decay over contiguous mini-batches in a seeded order."""
    n, _, Y, X = data.f0.shape
    nblocks = n // batch
    if nblocks < 1:
        raise ValueError("need at least one full batch")
    rng = np.random.default_rng(seed)
    order = rng.permutation(nblocks)
    B = net.buffers(batch, P, Y, X, True)
    stream = torch.cuda.current_stream()
    losses = []
    B.loss.zero_()
    for step in range(steps):
        if step % nblocks == 0 and step > 0:
            order = rng.permutation(nblocks)
        i0 = int(order[step % nblocks]) * batch
        K.make_input(batch, P, Y, X, data.f0[i0:i0 + batch], data.f1[i0:i0 + batch], B.inp, stream=stream)
        net.forward(B, stream)
        net.g32.zero_()
        net.backward(B, data.target[i0:i0 + batch], stream)
        a = step / max(1, steps - 1)
        net.adamw(lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * a)), stream=stream)
        if (step + 1) % log_every == 0 or step + 1 == steps:
            losses.append(float(B.loss.item()) / log_every if (step + 1) % log_every == 0 else
                          float(B.loss.item()) / ((step + 1) % log_every))
            B.loss.zero_()
            if log:
                log("step %d/%d loss %.4e" % (step + 1, steps, losses[-1]))
    torch.cuda.synchronize()
    return losses


def _cold_first_residual(seeds, side, P, nblobs, check_every=10, device="cuda") -> float:
    """Smallest residual of a cold start at its first check over the given pairs."""
    f0, f1 = make_pairs(seeds, side, nblobs, device)
    plan = Plan(rgb_grid(side, side, P), batch=1, stream=torch.cuda.current_stream().cuda_stream)
    r = min(plan.solve(f0[i:i + 1], f1[i:i + 1], check_every, 0.0, check_every=check_every).residual
            for i in range(len(seeds)))
    plan.close()
    return r


# (name, dual source, dual_support): "net" = the network's dual, "formula" = the fixed-point dual, "zero"
VARIANTS = (("net", "net", 0.0), ("zero", "zero", 0.0), ("formula", "formula", 0.3))


def _evaluate(net: UNet, seeds, side: int, P: int, nblobs: int, tol: float = 1e-4, max_iters: int = 10000,
              fallback: float = 0.0, ref_tol: float = 1e-6, ref_iters: int = 20000, check_every: int = 10,
              variants=VARIANTS, device="cuda", log=None) -> dict:
    """Cold vs warm starts on held-out pairs: iterations and wall time to `tol` (inference included),
    and the error of f at the stop against a reference solved to `ref_tol`.  Each variant is
    (name, dual_init, dual_support)."""
    stream = torch.cuda.current_stream()
    plan = Plan(rgb_grid(side, side, P), batch=1, stream=stream.cuda_stream)
    init = torch.empty(plan.path_size, dtype=torch.float32, device=device)
    dual = torch.empty(plan.dual_size, dtype=torch.float32, device=device)
    f_run = torch.empty((P - 1, 3, side, side), dtype=torch.float32, device=device)
    f_ref = torch.empty_like(f_run)
    rows = []
    # warm up the kernels, graphs and the network buffers once
    f0, f1 = make_pairs([seeds[0]], side, nblobs, device)
    net.predict(f0, f1, P, init, dual, stream)
    plan.solve(f0, f1, 2 * check_every, 0.0, check_every=check_every)
    plan.solve_warm(f0, f1, init, 2 * check_every, 0.0, check_every=check_every)
    torch.cuda.synchronize()

    def err():
        plan.path_into(f_run)
        return float(torch.linalg.vector_norm(f_run - f_ref)) / float(torch.linalg.vector_norm(f_ref))

    for s in seeds:
        f0, f1 = make_pairs([s], side, nblobs, device)
        ref = plan.solve(f0, f1, ref_iters, ref_tol, check_every=50)
        plan.path_into(f_ref)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cold = plan.solve(f0, f1, max_iters, tol, check_every=check_every)
        torch.cuda.synchronize()
        row = dict(seed=s, ref_iters=ref.iterations, ref_residual=ref.residual, cold_iters=cold.iterations,
                   cold_ms=(time.perf_counter() - t0) * 1e3, cold_converged=cold.converged, cold_err=err())
        for name, src, support in variants:
            t0 = time.perf_counter()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            net.predict(f0, f1, P, init, dual if src == "net" else None, stream)
            ev1.record(stream)
            w = plan.solve_warm(f0, f1, init, max_iters, tol, dual_init=src == "formula", dual_support=support,
                                fallback_residual=fallback, check_every=check_every,
                                init_dual=dual if src == "net" else None)
            torch.cuda.synchronize()
            row.update({name + "_iters": w.iterations, name + "_ms": (time.perf_counter() - t0) * 1e3,
                        name + "_infer_ms": ev0.elapsed_time(ev1), name + "_used_cold": w.used_cold,
                        name + "_converged": w.converged, name + "_err": err()})
        rows.append(row)
        if log:
            log("seed %d: cold %d it %.1f ms err %.1e | " % (s, row["cold_iters"], row["cold_ms"], row["cold_err"]) +
                " | ".join("%s %d it %.1f ms err %.1e%s" % (n, row[n + "_iters"], row[n + "_ms"], row[n + "_err"],
                                                          " [fallback]" if row[n + "_used_cold"] else "")
                           for n, _, _ in variants))
    plan.close()

    def stat(key):
        a = np.array([r[key] for r in rows], float)
        return {"mean": float(a.mean()), "p50": float(np.median(a)), "p90": float(np.percentile(a, 90))}

    out = {"pairs": len(rows), "tol": tol, "ref_tol": ref_tol,
           "cold": {"iters": stat("cold_iters"), "ms": stat("cold_ms"), "err": stat("cold_err"),
                    "all_converged": bool(all(r["cold_converged"] for r in rows))}}
    for n, src, support in variants:
        out[n] = {"dual": src, "dual_support": support, "iters": stat(n + "_iters"), "ms": stat(n + "_ms"),
                  "infer_ms": stat(n + "_infer_ms"), "err": stat(n + "_err"),
                  "fallbacks": int(sum(r[n + "_used_cold"] for r in rows)),
                  "all_converged": bool(all(r[n + "_converged"] for r in rows))}
    out["rows"] = rows
    return out


def solve_targets(*a, **k) -> PairSet:
    with side_stream():
        return _solve_targets(*a, **k)


def train(*a, **k) -> List[float]:
    with side_stream():
        return _train(*a, **k)


def cold_first_residual(*a, **k) -> float:
    with side_stream():
        return _cold_first_residual(*a, **k)


def evaluate(*a, **k) -> dict:
    with side_stream():
        return _evaluate(*a, **k)


def main(argv=None):
    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start")
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--P", type=int, default=32)
    ap.add_argument("--blobs", type=int, default=16)
    ap.add_argument("--train-pairs", type=int, default=2000)
    ap.add_argument("--eval-pairs", type=int, default=200)
    ap.add_argument("--eval-seed0", type=int, default=1_000_000)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--target-tol", type=float, default=1e-5)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--widths", type=str, default=",".join(map(str, WIDTHS)))
    ap.add_argument("--out", type=str, default="warmstart_report.json")
    ap.add_argument("--save", type=str, default="", help="write the trained weights (.npz)")
    ap.add_argument("--load", type=str, default="", help="skip training: evaluate saved weights")
    a = ap.parse_args(argv)
    torch.cuda.init()

    def log(msg):
        print("[warmstart] " + msg, flush=True)

    widths = tuple(int(w) for w in a.widths.split(","))
    t_data = t_train = 0.0
    losses: List[float] = []
    if a.load:
        net, meta = UNet.load(a.load)
        widths = net.widths
        log("loaded %s (%s)" % (a.load, meta))
    else:
        t0 = time.perf_counter()
        data = solve_targets(range(a.train_pairs), a.side, a.P, a.blobs, tol=a.target_tol, log=log)
        t_data = time.perf_counter() - t0
        log("targets: %.1f s, mean %.0f iterations" % (t_data, np.mean(data.iterations)))
        net = UNet(widths, seed=0)
        log("U-Net widths %s, %d parameters" % (widths, net.n_params))
        t0 = time.perf_counter()
        losses = train(net, data, a.P, a.steps, a.batch, a.lr, log=log)
        t_train = time.perf_counter() - t0
        del data
        torch.cuda.empty_cache()
        if a.save:
            net.save(a.save, side=a.side, P=a.P, blobs=a.blobs, train_pairs=a.train_pairs, steps=a.steps)
    fallback = cold_first_residual(range(8), a.side, a.P, a.blobs)
    log("fallback threshold (best cold first-check residual on training pairs): %.3e" % fallback)
    ev = evaluate(net, list(range(a.eval_seed0, a.eval_seed0 + a.eval_pairs)), a.side, a.P, a.blobs, tol=a.tol,
                  fallback=fallback, log=log)
    rep = {"config": {"side": a.side, "P": a.P, "blobs": a.blobs, "train_pairs": a.train_pairs,
                      "eval_pairs": a.eval_pairs, "steps": a.steps, "batch": a.batch, "lr": a.lr,
                      "widths": widths, "params": net.n_params, "target_tol": a.target_tol},
           "data_s": t_data, "train_s": t_train, "losses": losses, "fallback_residual": fallback, "eval": ev}
    with open(a.out, "w") as fh:
        json.dump(rep, fh, indent=1)
    for n, _, _ in VARIANTS:
        log("%s: cold %.0f it (p90 %.0f) %.1f ms err %.1e; warm %.0f it (p90 %.0f) %.1f ms err %.1e, fallbacks %d" % (
            n, ev["cold"]["iters"]["mean"], ev["cold"]["iters"]["p90"], ev["cold"]["ms"]["mean"],
            ev["cold"]["err"]["mean"], ev[n]["iters"]["mean"], ev[n]["iters"]["p90"], ev[n]["ms"]["mean"],
            ev[n]["err"]["mean"], ev[n]["fallbacks"]))
    return rep


if __name__ == "__main__":
    main()
