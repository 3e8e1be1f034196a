"""Warm-start network kernels (ot_nn_*) against the FP64 reference in
oracle/unet.py, on bf16-rounded inputs (GPU).

Tolerances: a convolution output accumulates K = 27 * Cin products in fp32;
its error is bounded by a small multiple of eps32 times the sum of |terms|,
so outputs are compared within 1e-5 * conv(|x|, |w|).  Outputs stored in
bf16 carry one more rounding of 2^-8 relative.  Weight gradients accumulate
over the voxels in fp32 and are compared the same way."""
import numpy as np
import pytest

from oracle import unet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_04840_gb300 import _build
    _build.build()
    from paper_1501_04840_gb300 import nn
    nn.lib()
    return nn


def _bf(shape, seed, scale=1.0):
    import torch
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(*shape, generator=g) * scale).to(torch.bfloat16)


def _np(t):
    import torch
    return t.detach().to("cpu", torch.float64).numpy()


BF_REL = 2.0 ** -8


@pytest.mark.parametrize("cin,cout,vol", [(16, 32, (2, 3, 5, 6)), (32, 24, (1, 4, 7, 9)), (48, 16, (1, 2, 8, 8)),
                                          (16, 8, (1, 3, 3, 11))])
def test_conv3d_forward_fp32(K, cin, cout, vol):
    import torch
    x = _bf(vol + (cin,), 1)
    w = _bf((cout, 27, cin), 2, 0.2)
    b = torch.randn(cout, generator=torch.Generator().manual_seed(3))
    y = torch.full(vol + (cout,), float("nan"), dtype=torch.float32, device="cuda")
    K.conv3d(vol, K.whole(x.cuda()), w.cuda(), b.cuda(), K.whole(y), relu=False, out_f32=True)
    torch.cuda.synchronize()
    ref = unet.conv3d(_np(x), _np(w), b.double().numpy())
    bound = unet.conv3d(np.abs(_np(x)), np.abs(_np(w))) + np.abs(b.double().numpy())
    assert np.all(np.abs(y.cpu().double().numpy() - ref) <= 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("cin,cout,vol,out_f32", [(16, 16, (1, 3, 8, 16), True), (32, 64, (2, 2, 5, 32), True),
                                                  (64, 48, (1, 2, 3, 128), False), (16, 32, (1, 4, 9, 64), False),
                                                  (48, 16, (2, 3, 4, 8), True), (16, 16, (2, 2, 3, 256), True),
                                                  (32, 64, (1, 2, 9, 128), False), (32, 32, (1, 2, 5, 128), True)])
def test_conv3d_tcgen05_tiles(K, cin, cout, vol, out_f32, monkeypatch):
    """Shapes the tcgen05 convolution takes (cout % 16 == 0, X dividing 128 or a multiple of it): tiles of
    128 voxels over one or several rows, partial tiles at the y edge, rows of 128 voxels (X = 128, 256) in
    the four-row block form (the default up to 64 output channels), the halo-row form (DYNOT_CONV=halo) and
    the per-tap form (DYNOT_CONV=tap), fp32 and bf16 outputs with ReLU, against the oracle; the mma.sync
    kernels (DYNOT_CONV=mma) give the same outputs within the same bound."""
    import torch
    x = _bf(vol + (cin,), 11)
    w = _bf((cout, 27, cin), 12, 0.2)
    b = torch.randn(cout, generator=torch.Generator().manual_seed(13))
    ref = unet.conv3d(_np(x), _np(w), b.double().numpy(), relu=True)
    bound = unet.conv3d(np.abs(_np(x)), np.abs(_np(w))) + np.abs(b.double().numpy())
    outs = []
    for kind in ("tcgen05", "halo", "tap", "mma"):
        monkeypatch.setenv("DYNOT_CONV", kind)
        dt = torch.float32 if out_f32 else torch.bfloat16
        y = torch.full(vol + (cout,), float("nan"), dtype=dt, device="cuda")
        K.conv3d(vol, K.whole(x.cuda()), w.cuda(), b.cuda(), K.whole(y), relu=True, out_f32=out_f32)
        torch.cuda.synchronize()
        K.check()
        got = y.cpu().double().numpy()
        rel = 0.0 if out_f32 else BF_REL
        assert np.all(np.abs(got - ref) <= rel * np.abs(ref) + 1e-5 * bound + 1e-30), kind
        outs.append(got)


@pytest.mark.parametrize("cin,cout,vol", [(16, 16, (4, 32, 40, 128)), (48, 16, (2, 32, 75, 128)),
                                          (16, 16, (2, 32, 45, 256))])
def test_conv3d_persistent_rows_equal_row_blocks(K, cin, cout, vol, monkeypatch):
    """The persistent form with one MMA per tap (DYNOT_CONV=persist) runs CTAs (two per SM) that
    walk the tiles with a two-stage copy ring and two accumulators in tensor memory, so that a tile's epilogue
    overlaps the next tile's MMAs.  Its MMAs are those of the one-tile-per-CTA row blocks (DYNOT_CONV=rows) in
    the same order: the outputs are equal bit for bit.  The volumes have 640 to 768 tiles, so every CTA
    reuses both accumulators several times, with a partial last row block."""
    import torch
    x = _bf(vol + (cin,), 31).cuda()
    w = _bf((cout, 27, cin), 32, 0.2).cuda()
    b = torch.randn(cout, generator=torch.Generator().manual_seed(33)).cuda()
    outs = []
    for kind in ("persist", "rows"):
        monkeypatch.setenv("DYNOT_CONV", kind)
        y = torch.full(vol + (cout,), float("nan"), dtype=torch.bfloat16, device="cuda")
        K.conv3d(vol, K.whole(x), w, b, K.whole(y), relu=True)
        torch.cuda.synchronize()
        K.check()
        outs.append(y)
    assert not torch.isnan(outs[0].float()).any()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("cin,cout,vol", [(16, 16, (4, 32, 40, 128)), (48, 16, (2, 32, 75, 128)),
                                          (16, 32, (2, 32, 42, 128)), (32, 32, (1, 32, 37, 256))])
def test_conv3d_stacked_taps_match_row_blocks(K, cin, cout, vol, monkeypatch):
    """With 16 and 32 output channels on rows of 128 voxels the convolution issues one MMA per input row and dx
    for the three dy taps together (N = 3 Cout), with persistent CTAs (one per SM) walking 640 to 704 tiles, so that every CTA
    reuses both accumulators; the first stage of a tile clears each row by its own tap.  fp32 outputs against
    the one-tile-per-CTA row blocks (DYNOT_CONV=rows), which sum the same products in another order: within
    2e-5 of the sum of absolute terms (each is within 1e-5 of the exact convolution)."""
    import torch
    x = _bf(vol + (cin,), 41).cuda()
    w = _bf((cout, 27, cin), 42, 0.2).cuda()
    b = torch.randn(cout, generator=torch.Generator().manual_seed(43)).cuda()
    outs = []
    for kind in ("tcgen05", "rows"):
        monkeypatch.setenv("DYNOT_CONV", kind)
        y = torch.full(vol + (cout,), float("nan"), dtype=torch.float32, device="cuda")
        K.conv3d(vol, K.whole(x), w, b, K.whole(y), relu=False, out_f32=True)
        torch.cuda.synchronize()
        K.check()
        outs.append(y)
    monkeypatch.setenv("DYNOT_CONV", "rows")
    bound = torch.empty(vol + (cout,), dtype=torch.float32, device="cuda")
    K.conv3d(vol, K.whole(x.abs()), w.abs(), b.abs(), K.whole(bound), relu=False, out_f32=True)
    torch.cuda.synchronize()
    assert not torch.isnan(outs[0]).any()
    assert bool(((outs[0] - outs[1]).abs() <= 2e-5 * bound + 1e-30).all())


def test_conv3d_slices_relu_bf16(K):
    """Input and output are channel slices of wider buffers; other channels stay untouched."""
    import torch
    vol = (2, 3, 6, 5)
    xb = _bf(vol + (48,), 4)
    w = _bf((16, 27, 16), 5, 0.3)
    b = torch.randn(16, generator=torch.Generator().manual_seed(6))
    yb = torch.full(vol + (40,), 7.0, dtype=torch.bfloat16, device="cuda")
    K.conv3d(vol, K.Slice(xb.cuda(), 16, 16), w.cuda(), b.cuda(), K.Slice(yb, 8, 16), relu=True)
    torch.cuda.synchronize()
    got = _np(yb)
    ref = unet.conv3d(_np(xb)[..., 16:32], _np(w), b.double().numpy(), relu=True)
    bound = unet.conv3d(np.abs(_np(xb)[..., 16:32]), np.abs(_np(w))) + np.abs(b.double().numpy())
    assert np.all(np.abs(got[..., 8:24] - ref) <= BF_REL * np.abs(ref) + 1e-5 * bound)
    assert np.all(got[..., :8] == 7.0) and np.all(got[..., 24:] == 7.0)


@pytest.mark.parametrize("cin,cout", [(16, 32), (48, 16), (24, 16)])
def test_conv3d_data_gradient(K, cin, cout):
    """dx = conv(dy, rotate(w)) equals the adjoint of the forward convolution."""
    import torch
    vol = (1, 3, 6, 7)
    dy = _bf(vol + (cout,), 7)
    w = _bf((cout, 27, cin), 8, 0.2)
    wr = torch.empty(cin * 27 * cout, dtype=torch.bfloat16, device="cuda")
    K.rotate_weights(cin, cout, w.cuda(), wr)
    dx = torch.empty(vol + (cin,), dtype=torch.float32, device="cuda")
    K.conv3d(vol, K.whole(dy.cuda()), wr, None, K.whole(dx), relu=False, out_f32=True)
    torch.cuda.synchronize()
    ref = unet.conv3d_dgrad(_np(dy), _np(w))
    bound = unet.conv3d_dgrad(np.abs(_np(dy)), np.abs(_np(w)))
    assert np.all(np.abs(dx.cpu().double().numpy() - ref) <= 1e-5 * bound + 1e-30)
    # the rotation itself is a permutation: exact
    wr_ref = np.transpose(_np(w)[:, ::-1, :], (2, 1, 0))
    assert np.array_equal(_np(wr).reshape(cin, 27, cout), wr_ref)


@pytest.mark.parametrize("cin,cout,vol", [(16, 32, (1, 4, 40, 40)), (32, 16, (2, 3, 9, 13))])
def test_conv3d_weight_gradient(K, cin, cout, vol):
    """dw and db accumulate (+=) over voxel chunks (several chunks of 4096 voxels, a ragged tail)."""
    import torch
    xb = _bf(vol + (cin + 16,), 9)
    dy = _bf(vol + (cout,), 10)
    dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    for _ in range(2):
        K.conv3d_wgrad(vol, K.Slice(xb.cuda(), 16, cin), K.whole(dy.cuda()), dw, db)
    torch.cuda.synchronize()
    x = _np(xb)[..., 16:]
    ref = 2 * unet.conv3d_wgrad(x, _np(dy))
    bound = 2 * unet.conv3d_wgrad(np.abs(x), np.abs(_np(dy)))
    assert np.all(np.abs(dw.cpu().double().numpy().reshape(cout, 27, cin) - ref) <= 1e-5 * bound + 1e-30)
    dbr = 2 * _np(dy).sum(axis=(0, 1, 2, 3))
    assert np.all(np.abs(db.cpu().double().numpy() - dbr) <= 1e-5 * 2 * np.abs(_np(dy)).sum(axis=(0, 1, 2, 3)))


@pytest.mark.parametrize("cin,cout,vol", [(16, 16, (2, 3, 7, 128)), (112, 48, (1, 4, 5, 128)),
                                          (48, 64, (1, 3, 6, 128)), (32, 32, (2, 2, 33, 128)),
                                          (32, 32, (2, 3, 9, 64)), (48, 48, (1, 4, 7, 32)), (64, 64, (2, 2, 6, 16)),
                                          (112, 48, (1, 3, 5, 32))])
def test_conv3d_weight_gradient_tcgen05(K, cin, cout, vol, monkeypatch):
    """Rows of 16 to 128 voxels take the tcgen05 weight gradient (dy as the M = 64 operand, the shifted input rows
    as N = Cin, both MN-major; 128 / X rows per stage; three dx accumulators per (dt, dy) pair; partial sums per
    chunk of row groups added in a fixed order): against the oracle, accumulated twice (+=), the input a channel
    slice of a wider tensor, row groups ragged at the y edge, from one CTA per SM (Cin = 112: 336 tensor-memory
    columns) to two; the mma.sync kernels (DYNOT_CONV=mma) agree."""
    import torch
    xb = _bf(vol + (cin + 16,), 51)
    dy = _bf(vol + (cout,), 52)
    x = _np(xb)[..., 16:]
    ref = 2 * unet.conv3d_wgrad(x, _np(dy))
    bound = 2 * unet.conv3d_wgrad(np.abs(x), np.abs(_np(dy)))
    for kind in ("tcgen05", "mma"):
        monkeypatch.setenv("DYNOT_CONV", kind)
        dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")
        for _ in range(2):
            K.conv3d_wgrad(vol, K.Slice(xb.cuda(), 16, cin), K.whole(dy.cuda()), dw, None)
        torch.cuda.synchronize()
        K.check()
        got = dw.cpu().double().numpy().reshape(cout, 27, cin)
        assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30), kind


def test_pool_upsample_relu_add(K):
    import torch
    vc = (2, 3, 4, 5)                  # coarse volume; fine is (2, 3, 8, 10)
    fine = _bf((2, 3, 8, 10, 16), 11)
    coarse = _bf(vc + (16,), 12)
    out_c = torch.empty(vc + (16,), dtype=torch.bfloat16, device="cuda")
    out_f = torch.empty((2, 3, 8, 10, 16), dtype=torch.bfloat16, device="cuda")
    K.pool(vc, K.whole(fine.cuda()), K.whole(out_c))
    ref = unet.round_bf16(unet.pool(_np(fine)))
    assert np.all(np.abs(_np(out_c) - ref) <= BF_REL * np.abs(ref))
    K.pool(vc, K.whole(coarse.cuda()), K.whole(out_f), backward=True)
    assert np.array_equal(_np(out_f), unet.pool_backward(_np(coarse)))      # quarter of a bf16: exact
    K.upsample(vc, K.whole(coarse.cuda()), K.whole(out_f))
    assert np.array_equal(_np(out_f), unet.upsample(_np(coarse)))
    K.upsample(vc, K.whole(fine.cuda()), K.whole(out_c), backward=True)
    ref = unet.upsample_backward(_np(fine))
    assert np.all(np.abs(_np(out_c) - ref) <= BF_REL * np.abs(ref))
    # relu backward masks where the stored activation is not positive (exact)
    g = _bf((2, 3, 8, 10, 16), 13).cuda()
    y = _bf((2, 3, 8, 10, 16), 14)
    gref = unet.relu_backward(_np(g), _np(y))
    K.relu_grad(K.whole(g), K.whole(y.cuda()))
    assert np.array_equal(_np(g), gref)
    # add into a slice
    a = _bf((2, 3, 8, 10, 16), 15)
    t = _bf((2, 3, 8, 10, 32), 16)
    tc = t.cuda()
    K.add_slice(K.whole(a.cuda()), K.Slice(tc, 16, 16))
    ref = unet.round_bf16(_np(t)[..., 16:] + _np(a))
    assert np.array_equal(_np(tc)[..., 16:], ref)
    assert np.array_equal(_np(tc)[..., :16], _np(t)[..., :16])


def test_mse_and_adamw(K):
    import torch
    rng = np.random.default_rng(17)
    out = torch.from_numpy(rng.standard_normal((300, 16)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.standard_normal((300, 12)).astype(np.float32)).to(torch.bfloat16).cuda()
    g = torch.empty((300, 16), dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    K.mse(out, 12, tgt, g, loss)
    torch.cuda.synchronize()
    lref, gref = unet.mse(out.cpu().double().numpy()[:, :12], _np(tgt))
    assert abs(loss.item() - lref) <= 1e-5 * lref
    gg = _np(g)
    assert np.all(np.abs(gg[:, :12] - gref) <= BF_REL * np.abs(gref) + 1e-12)
    assert not gg[:, 12:].any()
    # AdamW on fp32 master weights, 3 steps
    p = rng.standard_normal(1000).astype(np.float32)
    pt, mt, vt = torch.from_numpy(p.copy()).cuda(), torch.zeros(1000, device="cuda"), torch.zeros(1000, device="cuda")
    pb = torch.empty(1000, dtype=torch.bfloat16, device="cuda")
    pr, mr, vr = p.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in (1, 2, 3):
        gr = rng.standard_normal(1000).astype(np.float32)
        K.adamw(pt, torch.from_numpy(gr).cuda(), mt, vt, pb, 1e-2, 0.9, 0.999, 1e-8, 1e-2, step)
        pr, mr, vr = unet.adamw(pr, gr.astype(np.float64), mr, vr, 1e-2, 0.9, 0.999, 1e-8, 1e-2, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pt.cpu().double().numpy(), pr, rtol=1e-5, atol=1e-6)
    assert np.array_equal(_np(pb), unet.round_bf16(pt.cpu().numpy()))


def _expected_channels(P, Y, X, mx, my, mc, f, f0, f1):
    """Cell-aligned channels written from the paper's compact layout: m_x face x+1 (index x),
    m_y face y+1 (index y), colour face c+1 (periodic, index (c+1) % 3), f at time (t+1)/P."""
    ch = np.zeros((P, Y, X, 12))
    for c in range(3):
        ch[:, :, :X - 1, c] = mx[:, c]
        ch[:, :Y - 1, :, 3 + c] = my[:, c]
        ch[:, :, :, 6 + c] = mc[:, (c + 1) % 3]
        tau = (np.arange(1, P) / P)[:, None, None]
        ch[:P - 1, :, :, 9 + c] = f[:, c] - ((1 - tau) * f0[c] + tau * f1[c])
    return ch


def test_make_input_and_path_channels(K):
    import torch
    P, Y, X, N = 5, 6, 7, 2
    rng = np.random.default_rng(18)
    f0 = rng.random((N, 3, Y, X)).astype(np.float32)
    f1 = rng.random((N, 3, Y, X)).astype(np.float32)
    sc = np.array([2.0, 0.5], np.float32)
    inp = torch.empty((N, P, Y, X, 16), dtype=torch.bfloat16, device="cuda")
    K.make_input(N, P, Y, X, torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), inp,
                 scale=torch.from_numpy(sc).cuda())
    got = _np(inp)
    for n in range(N):
        a0 = np.transpose(f0[n], (1, 2, 0)).astype(np.float64) * sc[n]
        a1 = np.transpose(f1[n], (1, 2, 0)).astype(np.float64) * sc[n]
        for t in range(P):
            tau = (t + 1) / P
            ref = np.concatenate([a0, a1, (1 - tau) * a0 + tau * a1, np.full((Y, X, 1), (t + 0.5) / P),
                                  np.zeros((Y, X, 6))], axis=-1)
            assert np.all(np.abs(got[n, t] - ref) <= BF_REL * np.abs(ref) + 1e-7)
    # packed path -> channels (deviation of f from the interpolation) -> packed
    shapes = [(P, 3, Y, X - 1), (P, 3, Y - 1, X), (P, 3, Y, X), (P - 1, 3, Y, X)]
    parts = [[rng.standard_normal(s) for s in shapes] for _ in range(N)]
    packed = np.concatenate([np.concatenate([a.ravel() for a in pp]) for pp in parts]).astype(np.float32)
    pk = torch.from_numpy(packed).cuda()
    ch = torch.full((N, P, Y, X, 16), -5.0, dtype=torch.float32, device="cuda")
    d0, d1 = torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda()
    K.path_channels(N, Y, X, P, True, pk, ch, f0=d0, f1=d1)
    torch.cuda.synchronize()
    c = ch.cpu().double().numpy()
    for n in range(N):
        pp = [a.astype(np.float32).astype(np.float64) for a in parts[n]]
        ref = _expected_channels(P, Y, X, *pp, f0[n].astype(np.float64), f1[n].astype(np.float64))
        np.testing.assert_allclose(c[n, ..., :12], ref, rtol=0, atol=1e-6)
    assert np.all(c[..., 12:] == -5.0)
    back = torch.zeros_like(pk)
    K.path_channels(N, Y, X, P, False, back, ch, f0=d0, f1=d1)
    np.testing.assert_allclose(back.cpu().numpy(), packed, rtol=0, atol=1e-6)
    # without densities and with scale 1 the round trip is exact
    K.path_channels(N, Y, X, P, True, pk, ch)
    back.zero_()
    K.path_channels(N, Y, X, P, False, back, ch)
    assert np.array_equal(back.cpu().numpy(), packed)


def test_dual_channels(K):
    """Packed dual [n][k][t][c][y][x] <-> channels co + 3k + c: a permutation, exact both ways."""
    import torch
    N, P, Y, X = 2, 3, 5, 4
    rng = np.random.default_rng(19)
    packed = rng.standard_normal(N * 4 * P * 3 * Y * X).astype(np.float32)
    ch = torch.full((N, P, Y, X, 32), -3.0, device="cuda")
    pk = torch.from_numpy(packed).cuda()
    K.dual_channels(N, Y, X, P, True, pk, ch, 12)
    c = ch.cpu().numpy()
    ref = packed.reshape(N, 4, P, 3, Y, X).transpose(0, 2, 4, 5, 1, 3).reshape(N, P, Y, X, 12)
    assert np.array_equal(c[..., 12:24], ref)
    assert np.all(c[..., :12] == -3.0) and np.all(c[..., 24:] == -3.0)
    back = torch.zeros_like(pk)
    K.dual_channels(N, Y, X, P, False, back, ch, 12)
    assert np.array_equal(back.cpu().numpy(), packed)
