"""GPU parity: the CUDA path through the C-ABI against the CPU oracle on the
same seeded inputs.

Tolerances (binding for every comparison below):
  * integer coefficients Y, levels of the no-quantiser path, exact-integer
    reconstructions and SSE: bit-exact;
  * levels and samples of the quantised path: bit-exact against the oracle's
    binary32 decision path (same precision as the kernels).  Against float64:
    levels may differ by +-1 only where c / q lies within 2^-23 |c / q| of a
    rounding tie; samples reconstructed from the same levels may differ by +-1
    only where the float64 value lies within the binary32 error bound of the
    inverse network of a tie;
  * PSNR: within 1e-3 dB of the float64 definition.
"""
import math

import numpy as np
import pytest

from helpers import empty_like_img, from_dev, oracle_blocks, to_dev
from oracle import tx16_oracle as O
from paper_1606_07414_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1606_07414_gb300 import build, tx16

    build.build()
    tx16.load()
    return tx16


def _coeffs(n_blocks):
    import torch

    return torch.full((n_blocks * 256,), 0x7EADBEEF, dtype=torch.int32, device="cuda")


def _check_vs_fp64(levels_gpu, rec_gpu, ref, q):
    """Quantised path against the float64 definition: +-1 at near-ties only."""
    if q is None:
        return
    L64 = ref["levels64"]
    d = levels_gpu != L64
    assert np.all(np.abs(levels_gpu - L64) <= 1)
    c = np.abs(ref["c"][d])
    # c = Y s_u s_v / q carries two binary32 roundings on the GPU: |err| <= 2^-23 |c|
    assert np.all(np.abs(c - np.floor(c) - 0.5) <= 2.0 ** -23 * c + 1e-12)
    X64 = ref["X64"]
    d = rec_gpu != ref["recon64"]
    assert np.all(np.abs(rec_gpu.astype(np.int64) - ref["recon64"]) <= 1)
    frac = np.abs(X64[d]) % 1.0
    assert np.all(np.abs(frac - 0.5) <= ref["Xbound"][d])


# --------------------------------------------------------------------------
# Forward transform, bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,bits,pad", [((512, 512), 8, 0), ((48, 80), 8, 16), ((16, 16), 8, 0),
                                            ((16, 272), 8, 0), ((272, 16), 8, 32), ((64, 48), 10, 8),
                                            ((32, 528), 12, 0)])
def test_forward_bitexact(tx, shape, bits, pad):
    H, W = shape
    img = synth.ar1_image(100 + H + W + bits, H, W, 0.95, bits)
    d = to_dev(img, pad)
    nb = (H // 16) * (W // 16)
    co = _coeffs(nb)
    tx.tx16_forward([d], co, bits=bits)
    got = co.cpu().numpy().reshape(nb, 16, 16)
    want = O.forward_direct(O.image_to_blocks(img.astype(np.int64)))
    assert np.array_equal(got, want)


def test_forward_batch_mixed_sizes_and_depths(tx):
    """One call over images of uneven sizes, with 8- and 10-bit planes mixed
    (consecutive runs of one sample size share a launch)."""
    import torch

    sizes = [(32, 32, 8), (48, 1040, 8), (16, 16, 10), (64, 80, 10), (208, 16, 8), (16, 48, 8)]
    imgs = [synth.ar1_image(7 + i, h, w, 0.9, b) for i, (h, w, b) in enumerate(sizes)]
    keep = [to_dev(im) for im in imgs]  # descriptors hold raw pointers: keep tensors alive
    devs = [tx.image(t, b) for t, (_, _, b) in zip(keep, sizes)]
    nb = sum((h // 16) * (w // 16) for h, w, _ in sizes)
    co = _coeffs(nb)
    tx.tx16_forward(devs, co)
    torch.cuda.synchronize()
    got = co.cpu().numpy().reshape(nb, 16, 16)
    want = np.concatenate([O.forward_direct(O.image_to_blocks(im.astype(np.int64))) for im in imgs])
    assert np.array_equal(got, want)


def test_forward_extreme_values(tx):
    """Saturated and alternating planes reach the magnitude bound 256 (2^bits-1)."""
    for bits in (8, 12):
        peak = (1 << bits) - 1
        dt = np.uint8 if bits == 8 else np.uint16
        planes = [np.full((32, 32), peak, dt), np.zeros((32, 32), dt),
                  ((np.indices((32, 32)).sum(0) % 2) * peak).astype(dt),
                  np.tile(np.array(O.T[5] > 0, dt)[None, :] * peak, (32, 2)).astype(dt)]
        for p in planes:
            co = _coeffs(4)
            tx.tx16_forward([to_dev(p)], co, bits=bits)
            got = co.cpu().numpy().reshape(4, 16, 16)
            assert np.array_equal(got, O.forward_direct(O.image_to_blocks(p.astype(np.int64))))


# --------------------------------------------------------------------------
# Fused codec and the unfused form
# --------------------------------------------------------------------------
CASES = [(None, 1), (None, 16), (None, 150), (None, 256), (8.0, 4), (16.0, 16), (32.0, 64),
         (16.0, 256), (5.3, 100), (2.0 ** -8, 256)]


@pytest.mark.parametrize("q,r", CASES)
def test_codec_parity(tx, q, r):
    import torch

    H, W, bits = 80, 272, 8  # 85 blocks: 5 full tiles + a ragged tail of 5
    img = synth.ar1_image(1 + r, H, W, 0.95, bits)
    d = to_dev(img)
    out = empty_like_img(H, W, bits, pad=16)
    nb = (H // 16) * (W // 16)
    lev = _coeffs(nb)
    sse = torch.zeros(1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([d], [out], [(q, r)], sse=sse, levels=lev, bits=bits)
    torch.cuda.synchronize()
    ref = oracle_blocks(O.image_to_blocks(img.astype(np.int64)), q, r, bits)
    L = lev.cpu().numpy().reshape(nb, 16, 16)
    assert np.array_equal(L, ref["levels"])
    rec = O.image_to_blocks(from_dev(out, bits).astype(np.int64))
    assert np.array_equal(rec, ref["recon"])
    want_sse = O.sse(img, O.blocks_to_image(ref["recon"], H, W))
    assert int(sse.item()) == want_sse
    _check_vs_fp64(L, rec, ref, q)
    if q is not None:
        psnr64 = O.psnr(O.sse(img, O.blocks_to_image(ref["recon_def"], H, W)), H, W, bits)
        psnr_gpu = tx.tx16_psnr([int(sse.item())], [tx.image(d, bits)])[0]
        if math.isfinite(psnr64):
            assert abs(psnr_gpu - psnr64) < 1e-3
        else:
            assert psnr_gpu == psnr64


def test_config1_image(tx):
    """The paper's image experiment shape: one 512 x 512 AR(1) image (rho
    0.95, seed 1), r = 16 zig-zag coefficients, no quantiser; PSNR exact."""
    import torch

    img = synth.ar1_image(1, 512, 512, 0.95)
    d = to_dev(img)
    out = empty_like_img(512, 512, 8)
    sse = torch.zeros(1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([d], [out], [(None, 16)], sse=sse)
    ref = O.codec_image(img, None, 16, 8)
    assert np.array_equal(from_dev(out, 8), ref["recon"])
    assert int(sse.item()) == ref["sse"]
    assert tx.tx16_psnr([int(sse.item())], [tx.image(d)])[0] == pytest.approx(ref["psnr"], abs=1e-12)


def test_codec_batch_uneven_sizes_and_depths(tx):
    import torch

    spec = [(16, 16, 8, 8.0, 4), (96, 48, 8, None, 32), (48, 304, 10, 16.0, 64), (32, 32, 10, None, 256),
            (64, 64, 8, 32.0, 128), (16, 400, 8, 16.0, 8)]
    imgs, ins, outs, qp, keep = [], [], [], [], []
    for i, (h, w, b, q, r) in enumerate(spec):
        im = synth.ar1_image(40 + i, h, w, 0.85 + 0.02 * i, b)
        imgs.append(im)
        keep.append(to_dev(im))  # descriptors hold raw pointers: keep tensors alive
        ins.append(tx.image(keep[-1], b))
        o = empty_like_img(h, w, b)
        outs.append(o)
        qp.append((q, r))
    nb = sum((h // 16) * (w // 16) for h, w, *_ in spec)
    lev = _coeffs(nb)
    sse = torch.zeros(len(spec), dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch(ins, [tx.image(o, b) for o, (_, _, b, _, _) in zip(outs, spec)], qp, sse=sse,
                        levels=lev)
    torch.cuda.synchronize()
    L = lev.cpu().numpy().reshape(nb, 16, 16)
    k = 0
    for i, (h, w, b, q, r) in enumerate(spec):
        n = (h // 16) * (w // 16)
        ref = oracle_blocks(O.image_to_blocks(imgs[i].astype(np.int64)), q, r, b)
        assert np.array_equal(L[k:k + n], ref["levels"]), i
        rec = from_dev(outs[i], b)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(imgs[i], rec), i
        k += n


@pytest.mark.parametrize("q,r", [(None, 16), (16.0, 64), (8.0, 256)])
def test_unfused_form_equals_fused(tx, q, r):
    """forward -> quantise -> inverse -> sse (four launches) == codec (one)."""
    import torch

    H, W = 112, 208
    img = synth.ar1_image(77, H, W, 0.95)
    d = to_dev(img)
    nb = (H // 16) * (W // 16)
    co = _coeffs(nb)
    lev = _coeffs(nb)
    rec1 = empty_like_img(H, W, 8)
    rec2 = empty_like_img(H, W, 8)
    s1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    s2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    tx.tx16_forward([d], co)
    tx.tx16_quantise(co, nb, q, r, lev)
    tx.tx16_inverse(lev, [rec1], [(q, r)])
    tx.tx16_sse([d], [rec1], s1)
    lev2 = _coeffs(nb)
    tx.tx16_codec_batch([d], [rec2], [(q, r)], sse=s2, levels=lev2)
    torch.cuda.synchronize()
    assert torch.equal(lev, lev2)
    assert torch.equal(rec1, rec2)
    assert s1.item() == s2.item()
    # in-place quantisation (levels may alias coeffs)
    tx.tx16_quantise(co, nb, q, r, co)
    assert torch.equal(co, lev)


def test_codec_without_outputs_still_reduces(tx):
    import torch

    img = synth.ar1_image(5, 64, 64, 0.9)
    d = to_dev(img)
    sse = torch.zeros(1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([d], None, [(16.0, 16)], sse=sse)
    ref = O.codec_image(img, 16.0, 16, 8, "fp32")
    assert int(sse.item()) == ref["sse"]


def test_sse_is_reset_each_call(tx):
    import torch

    img = synth.ar1_image(6, 64, 64, 0.9)
    d = to_dev(img)
    sse = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    for _ in range(2):
        tx.tx16_codec_batch([d], None, [(None, 8)], sse=sse)
    assert int(sse.item()) == O.codec_image(img, None, 8, 8)["sse"]


def test_wide_and_tall_images(tx):
    """One block row 16 x 65536 (4096 blocks) and one block column."""
    import torch

    for H, W in ((16, 65536), (4096, 16)):
        img = synth.ar1_image(9, H, W, 0.95)
        d = to_dev(img)
        out = empty_like_img(H, W, 8)
        sse = torch.zeros(1, dtype=torch.int64, device="cuda")
        tx.tx16_codec_batch([d], [out], [(16.0, 16)], sse=sse)
        ref = O.codec_image(img, 16.0, 16, 8, "fp32")
        assert np.array_equal(from_dev(out, 8), ref["recon"])
        assert int(sse.item()) == ref["sse"]


# --------------------------------------------------------------------------
# Codec without level output: several images per launch, tiles that straddle
# images, and batches large enough that every warp codes tiles of several
# images in turn.  A batch with fewer 32-block warp tiles than the GPU has
# SMs runs on the two-blocks-per-pair kernel; a larger one on the
# one-block-per-thread kernel (every zonal class).  `repeat` copies of the
# set of shapes give both: 1 copy (25 warp tiles) the pair kernel, 20 copies
# (500 warp tiles) the one-block-per-thread kernel.
# --------------------------------------------------------------------------
NOLEV_CASES = [(16.0, 8), (None, 8), (16.0, 16), (None, 16), (12.0, 32), (None, 32), (16.0, 64), (None, 64),
               (16.0, 128), (None, 100), (8.0, 200), (None, 256)]


@pytest.mark.parametrize("repeat", [1, 20])
@pytest.mark.parametrize("q,r", NOLEV_CASES)
def test_codec_without_levels_batch(tx, q, r, repeat):
    import torch

    shapes = [(16, 16), (80, 272), (48, 528), (16, 512), (160, 640), (32, 32), (32, 48), (64, 16)] * repeat
    imgs = [synth.ar1_image(700 + i + r, h, w, 0.9 + 0.01 * (i % 8), 8) for i, (h, w) in enumerate(shapes)]
    keep = [to_dev(im) for im in imgs]
    outs = [empty_like_img(h, w, 8, pad=16) for h, w in shapes]
    sse = torch.full((len(imgs),), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d) for d in keep], [tx.image(o) for o in outs], [(q, r)] * len(imgs), sse=sse)
    torch.cuda.synchronize()
    for i, (im, (h, w)) in enumerate(zip(imgs, shapes)):
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, 8)
        rec = from_dev(outs[i], 8)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i


@pytest.mark.parametrize("q,r,frames", [(16.0, 16, 8), (None, 32, 5), (16.0, 8, 10)])
def test_codec_without_levels_many_tiles(tx, q, r, frames):
    """1920 x 1088 frames, enough tiles that each warp moves across images.
    Sampled blocks (every tile edge of the first and last frames, and 400
    random blocks of each frame) against the oracle; each frame's SSE
    against the sum over the GPU's own reconstruction."""
    import torch

    H, W = 1088, 1920
    fr = synth.video_frames(77 + r, frames, H, W, rho=0.95)
    d_in = torch.from_numpy(fr).cuda()
    d_out = torch.zeros_like(d_in)
    sse = torch.full((frames,), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d_in[i]) for i in range(frames)], [tx.image(d_out[i]) for i in range(frames)],
                        [(q, r)] * frames, sse=sse)
    torch.cuda.synchronize()
    rec = d_out.cpu().numpy()
    s = sse.cpu().numpy()
    nbx, nb = W // 16, (H // 16) * (W // 16)
    rng = np.random.default_rng(r)
    for i in range(frames):
        assert int(s[i]) == O.sse(fr[i], rec[i]), i
        pick = set(rng.integers(0, nb, 400).tolist())
        if i in (0, frames - 1):
            pick |= {b for t in range(0, nb, 32) for b in (t, t + 31) if b < nb}
            pick |= {nb - 1}
        pick = np.array(sorted(pick))
        X = np.stack([fr[i][(b // nbx) * 16:(b // nbx) * 16 + 16, (b % nbx) * 16:(b % nbx) * 16 + 16] for b in pick])
        got = np.stack([rec[i][(b // nbx) * 16:(b // nbx) * 16 + 16, (b % nbx) * 16:(b % nbx) * 16 + 16] for b in pick])
        ref = oracle_blocks(X.astype(np.int64), q, r, 8)
        assert np.array_equal(got, ref["recon"]), i


# --------------------------------------------------------------------------
# 9..12-bit planes through the fused path (one block per thread, 16-bit
# samples; a quantiser of q >= 2^(bits-8)/256, up to 8 kept columns, no
# levels) and the general kernel beside it
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bits,q,r", [(10, 16.0, 16), (10, 4.0, 8), (10, 64.0, 32), (12, 64.0, 16),
                                      (12, 16.0, 4), (9, 8.0, 16), (10, 2.0 ** -5, 16)])
def test_codec_16bit_without_levels(tx, bits, q, r):
    import torch

    shapes = [(80, 272), (16, 16), (64, 528), (48, 48)]
    imgs = [synth.ar1_image(900 + i + bits + r, h, w, 0.93, bits) for i, (h, w) in enumerate(shapes)]
    keep = [to_dev(im) for im in imgs]
    outs = [empty_like_img(h, w, bits, pad=8) for h, w in shapes]
    sse = torch.full((len(imgs),), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d, bits) for d in keep], [tx.image(o, bits) for o in outs],
                        [(q, r)] * len(imgs), sse=sse)
    torch.cuda.synchronize()
    for i, im in enumerate(imgs):
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, bits)
        rec = from_dev(outs[i], bits)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i


def test_codec_16bit_2160p_frame(tx):
    """One 3840 x 2160 10-bit frame (the serving mix's large request) through
    the fused 16-bit path: sampled blocks against the oracle, SSE against the
    GPU's own reconstruction."""
    import torch

    H, W, bits = 2160, 3840, 10
    img = synth.ar1_image(2160, H, W, 0.95, bits)
    d = to_dev(img)
    out = empty_like_img(H, W, bits)
    sse = torch.zeros(1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d, bits)], [tx.image(out, bits)], [(16.0, 16)], sse=sse)
    torch.cuda.synchronize()
    rec = from_dev(out, bits)
    assert int(sse.item()) == O.sse(img, rec)
    nbx, nb = W // 16, (H // 16) * (W // 16)
    rng = np.random.default_rng(10)
    pick = np.unique(np.concatenate([rng.integers(0, nb, 600), np.arange(0, nb, 32), [nb - 1]]))
    X = np.stack([img[(b // nbx) * 16:(b // nbx) * 16 + 16, (b % nbx) * 16:(b % nbx) * 16 + 16] for b in pick])
    got = np.stack([rec[(b // nbx) * 16:(b // nbx) * 16 + 16, (b % nbx) * 16:(b % nbx) * 16 + 16] for b in pick])
    ref = oracle_blocks(X.astype(np.int64), 16.0, 16, bits)
    assert np.array_equal(got, ref["recon"])


# --------------------------------------------------------------------------
# Clamping at both ends of the sample range: planes of extreme samples whose
# zonal reconstructions overshoot far below 0 and above the peak (Gibbs-like
# ringing), through the one-block-per-thread kernels (no levels, a batch of
# at least one warp tile per SM: `repeat` = 30 copies of the seven planes,
# 210 warp tiles), the pair kernel (levels requested, or the seven planes
# alone) and the 16-bit path
# --------------------------------------------------------------------------
def _extreme_planes(bits):
    peak = (1 << bits) - 1
    dt = np.uint8 if bits == 8 else np.uint16
    ii, jj = np.indices((64, 96))
    rng = np.random.default_rng(bits)
    planes = [((ii + jj) % 2) * peak,                      # checkerboard
              ((jj // 3) % 2) * peak,                      # vertical stripes, 3 wide
              ((ii // 2) % 2) * peak,                      # horizontal stripes, 2 wide
              (jj >= 45) * peak,                           # step edge inside a block
              rng.integers(0, 2, (64, 96)) * peak,         # random two-level
              np.full((64, 96), peak), np.zeros((64, 96))]
    return [p.astype(dt) for p in planes]


@pytest.mark.parametrize("q,r,levels,repeat", [(None, 32, False, 30), (None, 16, False, 30), (64.0, 4, False, 30),
                                               (64.0, 16, False, 30), (16.0, 32, False, 30), (64.0, 64, False, 30),
                                               (32.0, 128, False, 30), (24.0, 256, False, 30), (64.0, 16, False, 1),
                                               (8.0, 16, True, 1), (64.0, 64, False, 1), (32.0, 256, True, 1),
                                               (None, 150, True, 1)])
def test_codec_extreme_planes_clamp(tx, q, r, levels, repeat):
    import torch

    planes = _extreme_planes(8) * repeat
    keep = [to_dev(p) for p in planes]
    outs = [empty_like_img(64, 96, 8, pad=16) for _ in planes]
    sse = torch.full((len(planes),), -1, dtype=torch.int64, device="cuda")
    lev = _coeffs(len(planes) * 24) if levels else None
    tx.tx16_codec_batch([tx.image(d) for d in keep], [tx.image(o) for o in outs], [(q, r)] * len(planes),
                        sse=sse, levels=lev)
    torch.cuda.synchronize()
    overshoot = 0
    for i, im in enumerate(planes):
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, 8)
        rec = from_dev(outs[i], 8)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i
        overshoot += int(np.sum((ref["X64"] < -0.5) | (ref["X64"] > 255.5)))
    assert overshoot > 0  # the clamps were exercised


@pytest.mark.parametrize("bits,q,r", [(10, 64.0, 4), (10, 16.0, 16), (12, 64.0, 32), (9, 8.0, 16)])
def test_codec_16bit_extreme_planes_clamp(tx, bits, q, r):
    import torch

    planes = _extreme_planes(bits)
    keep = [to_dev(p) for p in planes]
    outs = [empty_like_img(64, 96, bits, pad=8) for _ in planes]
    sse = torch.full((len(planes),), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d, bits) for d in keep], [tx.image(o, bits) for o in outs],
                        [(q, r)] * len(planes), sse=sse)
    torch.cuda.synchronize()
    for i, im in enumerate(planes):
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, bits)
        rec = from_dev(outs[i], bits)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i


@pytest.mark.parametrize("q,r", [(16.0, 16), (None, 8), (12.0, 32)])
def test_codec_without_levels_ragged_many_images(tx, q, r):
    """64 images of 80 x 272 (85 blocks each: two full 32-block warp tiles and
    a ragged third), 5440 blocks in all: enough warp tiles for the
    one-block-per-thread kernel, whose warps then cross image boundaries and
    code ragged tails.  Every image bit-exact against the oracle."""
    import torch

    n, H, W = 64, 80, 272
    imgs = [synth.ar1_image(5000 + i + r, H, W, 0.8 + 0.003 * i, 8) for i in range(n)]
    keep = [to_dev(im) for im in imgs]
    outs = [empty_like_img(H, W, 8, pad=16) for _ in range(n)]
    sse = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d) for d in keep], [tx.image(o) for o in outs], [(q, r)] * n, sse=sse)
    torch.cuda.synchronize()
    X = np.concatenate([O.image_to_blocks(im.astype(np.int64)) for im in imgs])
    ref = oracle_blocks(X, q, r, 8)["recon"]
    got = np.concatenate([O.image_to_blocks(from_dev(o, 8).astype(np.int64)) for o in outs])
    assert np.array_equal(got, ref)
    for i in range(n):
        assert int(sse[i].item()) == O.sse(imgs[i], from_dev(outs[i], 8)), i


def test_codec_batch_mixed_classes_grouped(tx):
    """One tx16_codec_batch call (no levels) over images of every zonal class
    interleaved, large enough for the one-block-per-thread kernel: the library
    runs one launch per class, each image adding into its own SSE slot."""
    import torch

    rs = [4, 256, 16, 100, 32, 64, 8, 150, 1]
    qs = [16.0, None, 8.0, 32.0]
    shapes = [(80, 272), (48, 528), (160, 640), (32, 48), (64, 16)] * 12  # 223 warp tiles
    imgs = [synth.ar1_image(4100 + i, h, w, 0.9 + 0.01 * (i % 8), 8) for i, (h, w) in enumerate(shapes)]
    qp = [(qs[i % 4], rs[i % 9]) for i in range(len(imgs))]
    keep = [to_dev(im) for im in imgs]
    outs = [empty_like_img(h, w, 8, pad=16) for h, w in shapes]
    sse = torch.full((len(imgs),), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d) for d in keep], [tx.image(o) for o in outs], qp, sse=sse)
    torch.cuda.synchronize()
    for i, (im, (q, r)) in enumerate(zip(imgs, qp)):
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, 8)
        rec = from_dev(outs[i], 8)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i
