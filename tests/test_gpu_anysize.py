"""GPU parity of tx16_codec_any_size: images whose sides are not multiples of
16 (edge replication to whole blocks, only the image's own samples written
and counted) and colour images coded plane by plane, against the oracle's
``codec_image_any_size`` / ``codec_colour`` on the same seeded inputs.

Tolerance: bit-exact samples and SSE (the oracle takes the binary32 decision
path for q > 0, the exact-integer path otherwise, as the kernels do)."""
import numpy as np
import pytest

from oracle import tx16_oracle as O
from paper_1606_07414_gb300 import synth

pytestmark = pytest.mark.gpu

SENTINEL = 0x5A


@pytest.fixture(scope="module")
def tx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1606_07414_gb300 import build, tx16

    build.build()
    tx16.load()
    return tx16


def _pitch_samples(W: int, bits: int, extra: int = 0) -> int:
    """Smallest row length (samples) whose byte pitch is a multiple of 16."""
    per = 16 if bits == 8 else 8
    return -(-W // per) * per + extra


def _dev(img: np.ndarray, bits: int, extra: int = 0):
    import torch

    H, W = img.shape
    a = img.view(np.int16) if bits > 8 else img
    P = _pitch_samples(W, bits, extra)
    t = torch.full((H + 2, P), SENTINEL, dtype=torch.uint8 if bits == 8 else torch.int16, device="cuda")
    t[:H, :W] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t, t[:H, :W]


def _out(H: int, W: int, bits: int, extra: int = 0):
    import torch

    P = _pitch_samples(W, bits, extra)
    t = torch.full((H + 2, P), SENTINEL, dtype=torch.uint8 if bits == 8 else torch.int16, device="cuda")
    return t, t[:H, :W]


def _host(t, bits: int) -> np.ndarray:
    a = t.cpu().contiguous().numpy()
    return a.view(np.uint16) if bits > 8 else a


def _oracle(img, q, r, bits):
    if q is None:
        return O.codec_image_any_size(img, None, r, bits)
    return O.codec_image_any_size(img, float(np.float32(q)), r, bits, "fp32")


def _run(tx, imgs, qps, bits_list, extra=0):
    import torch

    keep, ins, outs, fulls = [], [], [], []
    for img, bits in zip(imgs, bits_list):
        full_in, v_in = _dev(img, bits, extra)
        full_out, v_out = _out(*img.shape, bits, extra)
        keep += [full_in, full_out]
        ins.append(tx.image(v_in, bits))
        outs.append(tx.image(v_out, bits))
        fulls.append(full_out)
    sse = torch.full((len(imgs),), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_any_size(ins, outs, qps, sse)
    torch.cuda.synchronize()
    # keep: the device buffers the returned descriptors point into
    return [_host(f, b) for f, b in zip(fulls, bits_list)], sse.cpu().numpy(), ins, keep


CASES = [
    # (H, W, bits, q, r)
    ((37, 50), 8, 16.0, 16),
    ((1, 1), 8, None, 256),
    ((1, 1), 8, 16.0, 1),
    ((15, 17), 8, 5.3, 64),
    ((500, 512), 8, 8.0, 64),     # ragged bottom only
    ((512, 500), 8, None, 16),    # ragged right only
    ((33, 17), 10, 4.0, 32),
    ((17, 40), 12, None, 8),      # 16-bit, last block 8 wide: tight pitch
    ((21, 9), 12, 2.0, 256),
    ((48, 64), 8, 16.0, 16),      # whole blocks
    ((100, 64), 8, 16.0, 128),    # ragged bottom, class E
    ((40, 48), 8, None, 256),     # ragged bottom, class F, no quantiser
    ((45, 70), 8, 8.0, 100),      # ragged both ways, class E
]


@pytest.mark.parametrize("shape,bits,q,r", CASES)
def test_any_size_bitexact(tx, shape, bits, q, r):
    H, W = shape
    img = synth.ar1_image(700 + H * 3 + W + bits, H, W, 0.95, bits)
    fulls, sse, _, _ = _run(tx, [img], [(q, r)], [bits])
    want = _oracle(img, q, r, bits)
    got = fulls[0]
    assert np.array_equal(got[:H, :W], want["recon"])
    assert int(sse[0]) == int(want["sse"])
    # nothing written outside the image: pitch padding and the rows below
    assert np.all(got[:H, W:] == SENTINEL)
    assert np.all(got[H:, :] == SENTINEL)


def test_1080p_frame_ragged_height(tx):
    """A real 1920 x 1080 frame: 1080 = 67.5 blocks, the last block row is
    half image, half replicated."""
    H, W = 1080, 1920
    img = synth.ar1_image(4242, H, W, 0.95, 8)
    fulls, sse, ins, keep = _run(tx, [img], [(16.0, 16)], [8])
    want = _oracle(img, 16.0, 16, 8)
    assert np.array_equal(fulls[0][:H, :W], want["recon"])
    assert int(sse[0]) == int(want["sse"])
    p = tx.tx16_psnr([int(sse[0])], ins)[0]
    assert abs(p - want["psnr"]) < 1e-9


def test_mixed_batch_and_depths(tx):
    """One call over images of different sizes, depths and quantisers (runs
    of equal sample size are split by the library)."""
    shapes = [(37, 50), (64, 64), (19, 300), (70, 33), (16, 17)]
    bits = [8, 10, 8, 12, 8]
    qps = [(16.0, 16), (None, 32), (3.0, 100), (8.0, 8), (None, 256)]
    imgs = [synth.ar1_image(900 + i, h, w, 0.9, b) for i, ((h, w), b) in enumerate(zip(shapes, bits))]
    fulls, sse, _, _ = _run(tx, imgs, qps, bits, extra=16)
    for i, (img, (q, r), b) in enumerate(zip(imgs, qps, bits)):
        H, W = img.shape
        want = _oracle(img, q, r, b)
        assert np.array_equal(fulls[i][:H, :W], want["recon"]), i
        assert int(sse[i]) == int(want["sse"]), i
        assert np.all(fulls[i][:H, W:] == SENTINEL)


def test_colour_planes(tx):
    """Colour image: three planes, each coded separately (same q: the
    oracle's codec_colour; then a coarser quantiser on two planes)."""
    H, W = 45, 70
    planes = [synth.ar1_image(1300 + c, H, W, 0.95, 8) for c in range(3)]
    fulls, sse, _, _ = _run(tx, planes, [(12.0, 32)] * 3, [8] * 3)
    want = O.codec_colour(planes, float(np.float32(12.0)), 32, 8, "fp32")
    for c in range(3):
        assert np.array_equal(fulls[c][:H, :W], want[c]["recon"])
        assert int(sse[c]) == int(want[c]["sse"])
    qps = [(8.0, 64), (24.0, 16), (24.0, 16)]
    fulls, sse, _, _ = _run(tx, planes, qps, [8] * 3)
    for c in range(3):
        w = _oracle(planes[c], *qps[c], 8)
        assert np.array_equal(fulls[c][:H, :W], w["recon"])
        assert int(sse[c]) == int(w["sse"])


def test_whole_blocks_match_codec_batch(tx):
    """On images with sides that are multiples of 16 the any-size entry gives
    tx16_codec_batch's samples and SSE."""
    import torch

    img = synth.ar1_image(77, 208, 320, 0.95, 8)
    fulls, sse, ins, keep = _run(tx, [img], [(16.0, 16)], [8])
    out = torch.zeros((208, 320), dtype=torch.uint8, device="cuda")
    s2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch(ins, [tx.image(out, 8)], [(16.0, 16)], s2)
    torch.cuda.synchronize()
    assert np.array_equal(fulls[0][:208, :320], out.cpu().numpy())
    assert int(sse[0]) == int(s2.cpu()[0])


def test_rejects_bad_arguments(tx):
    import torch

    t = torch.zeros((20, 48), dtype=torch.uint8, device="cuda")
    good = tx.image(t[:, :37], 8)
    bad_pitch = tx.tx16_image(t.data_ptr(), 37, 20, 40, 8)   # pitch not a multiple of 16
    short_pitch = tx.tx16_image(t.data_ptr(), 37, 20, 32, 8)  # pitch < width
    zero_w = tx.tx16_image(t.data_ptr(), 0, 20, 48, 8)
    for d in (bad_pitch, short_pitch, zero_w):
        with pytest.raises(tx.Tx16Error):
            tx.tx16_codec_any_size([d], None, [(16.0, 16)])
    other = tx.image(t[:, :36], 8)  # output width differs
    with pytest.raises(tx.Tx16Error):
        tx.tx16_codec_any_size([good], [other], [(16.0, 16)])
    tx.tx16_codec_any_size([], None, [])  # empty batch: no work, no error
