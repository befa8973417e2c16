"""GPU parity of tx16_codec_mixed (mixed 8/16 tiling with T and T8) against
the oracle's ``codec_image_mixed`` on the same seeded inputs.

Tolerance: bit-exact samples, split map and SSE.  The oracle takes its
rounding decisions in binary32 (precision 'fp32') for q > 0 and in exact
integers without a quantiser, as the kernel does; the tiling decision
compares exact integer squared errors."""
import numpy as np
import pytest

from helpers import empty_like_img, from_dev, to_dev
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


def _oracle(img, q, r16, r8, bits, mode):
    if q is None:
        return O.codec_image_mixed(img, None, r16, r8, bits, mode)
    return O.codec_image_mixed(img, float(np.float32(q)), r16, r8, bits, mode, "fp32")


def _run(tx, imgs, qps, bits_list):
    import torch

    keep = [to_dev(im) for im in imgs]
    outs = [empty_like_img(*im.shape, b, pad=16) for im, b in zip(imgs, bits_list)]
    nreg = sum((im.shape[0] // 16) * (im.shape[1] // 16) for im in imgs)
    split = torch.full((nreg,), 7, dtype=torch.uint8, device="cuda")
    sse = torch.full((len(imgs),), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_mixed([tx.image(d, b) for d, b in zip(keep, bits_list)],
                        [tx.image(o, b) for o, b in zip(outs, bits_list)], qps, split=split, sse=sse)
    torch.cuda.synchronize()
    return [from_dev(o, b) for o, b in zip(outs, bits_list)], split.cpu().numpy(), sse.cpu().numpy()


CASES = [(16.0, 16, 4, "auto"), (None, 16, 4, "auto"), (8.0, 64, 16, "auto"), (32.0, 4, 1, "auto"),
         (16.0, 16, 4, "16"), (16.0, 16, 4, "8"), (None, 256, 64, "8"), (5.3, 100, 30, "auto")]


@pytest.mark.parametrize("q,r16,r8,mode", CASES)
def test_mixed_bitexact(tx, q, r16, r8, mode):
    img = synth.ar1_image(300 + r16 + r8, 80, 272, 0.93, 8)
    recs, split, sse = _run(tx, [img], [(q, r16, r8, mode)], [8])
    want = _oracle(img, q, r16, r8, 8, mode)
    assert np.array_equal(recs[0], want["recon"])
    assert np.array_equal(split.astype(bool), want["split"].ravel())
    assert int(sse[0]) == want["sse"]
    if mode == "auto":
        assert 0 < int(split.sum()) < split.size or q is None or r16 == 4  # both tilings occur


# One case per compiled class pair of the one-region-per-thread kernel
# (16x16 class, 8x8 class): (A, 0), (B, 0), (B, 1), (C, 1), (D, 1); the image
# is 5 x 17 regions, so the last warp tile of 32 regions is ragged.
PAIR_CASES = [(12.0, 8, 4, "auto"), (16.0, 13, 3, "auto"), (10.0, 12, 16, "auto"), (7.0, 32, 9, "auto"),
              (8.0, 50, 12, "auto"), (1.0 / 256, 16, 4, "auto"), (200.0, 64, 16, "auto"), (9.0, 30, 10, "8")]


@pytest.mark.parametrize("q,r16,r8,mode", PAIR_CASES)
def test_mixed_pairs_bitexact(tx, q, r16, r8, mode):
    img = synth.ar1_image(900 + r16 * 3 + r8, 80, 272, 0.93, 8)
    recs, split, sse = _run(tx, [img], [(q, r16, r8, mode)], [8])
    want = _oracle(img, q, r16, r8, 8, mode)
    assert np.array_equal(recs[0], want["recon"])
    assert np.array_equal(split.astype(bool), want["split"].ravel())
    assert int(sse[0]) == want["sse"]


def test_mixed_batch_across_kernels(tx):
    """One call whose images go to different class pairs of the
    one-region-per-thread kernel and to the general kernel (no quantiser,
    r16 > 64, 10-bit), interleaved: each image's split-map range and SSE slot
    must be its own."""
    qps = [(16.0, 16, 4, "auto"), (None, 16, 4, "auto"), (7.0, 32, 9, "auto"), (5.0, 100, 8, "auto"),
           (12.0, 8, 2, "auto"), (3.0, 20, 40, "auto"), (16.0, 16, 4, "16"), (8.0, 64, 16, "auto")]
    shapes = [(48, 64), (32, 96), (64, 48), (16, 32), (80, 16), (32, 32), (48, 48), (16, 16)]
    bits = [8, 8, 8, 8, 8, 10, 8, 8]
    imgs = [synth.ar1_image(950 + i, h, w, 0.9, b) for i, ((h, w), b) in enumerate(zip(shapes, bits))]
    recs, split, sse = _run(tx, imgs, qps, bits)
    k = 0
    for i, (im, (q, r16, r8, mode), b) in enumerate(zip(imgs, qps, bits)):
        want = _oracle(im, q, r16, r8, b, mode)
        n = want["split"].size
        assert np.array_equal(recs[i], want["recon"]), i
        assert np.array_equal(split[k:k + n].astype(bool), want["split"].ravel()), i
        assert int(sse[i]) == want["sse"], i
        k += n


def test_mixed_more_images_than_one_launch(tx):
    """170 images of one class pair: more than one launch's worth of image
    descriptors."""
    n = 170
    imgs = [synth.ar1_image(2000 + i, 16 * (1 + i % 3), 32, 0.9, 8) for i in range(n)]
    qps = [(8.0 + (i % 5), 16, 4, "auto") for i in range(n)]
    recs, split, sse = _run(tx, imgs, qps, [8] * n)
    k = 0
    for i, (im, (q, r16, r8, mode)) in enumerate(zip(imgs, qps)):
        want = _oracle(im, q, r16, r8, 8, mode)
        m = want["split"].size
        assert np.array_equal(recs[i], want["recon"]), i
        assert np.array_equal(split[k:k + m].astype(bool), want["split"].ravel()), i
        assert int(sse[i]) == want["sse"], i
        k += m


def test_mixed_without_output_plane(tx):
    """No output plane: the split map and SSE alone (general kernel)."""
    import torch

    img = synth.ar1_image(960, 64, 96, 0.93, 8)
    d = to_dev(img)
    split = torch.full((24,), 7, dtype=torch.uint8, device="cuda")
    sse = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_mixed([tx.image(d)], None, [(16.0, 16, 4, "auto")], split=split, sse=sse)
    torch.cuda.synchronize()
    want = _oracle(img, 16.0, 16, 4, 8, "auto")
    assert np.array_equal(split.cpu().numpy().astype(bool), want["split"].ravel())
    assert int(sse.cpu().numpy()[0]) == want["sse"]


def test_mixed_lossless_and_flat(tx):
    """r16 = 256, r8 = 64, no quantiser: lossless whichever tiling; a flat
    image ties everywhere and stays 16x16."""
    img = synth.ar1_image(301, 48, 64, 0.9, 8)
    recs, split, sse = _run(tx, [img], [(None, 256, 64, "auto")], [8])
    assert np.array_equal(recs[0], img) and int(sse[0]) == 0 and not split.any()
    flat = np.full((32, 48), 91, dtype=np.uint8)
    recs, split, sse = _run(tx, [flat], [(None, 1, 1, "auto")], [8])
    assert np.array_equal(recs[0], flat) and not split.any() and int(sse[0]) == 0


def test_mixed_batch_depths(tx):
    shapes = [(48, 64), (32, 32), (64, 48), (16, 16)]
    bits = [8, 10, 8, 12]
    qps = [(16.0, 16, 4, "auto"), (4.0, 32, 8, "auto"), (None, 16, 4, "8"), (64.0, 8, 2, "auto")]
    imgs = [synth.ar1_image(310 + i, h, w, 0.9, b) for i, ((h, w), b) in enumerate(zip(shapes, bits))]
    recs, split, sse = _run(tx, imgs, qps, bits)
    k = 0
    for i, (im, (q, r16, r8, mode), b) in enumerate(zip(imgs, qps, bits)):
        qq = q * (1 << (b - 8)) if q is not None else None
        want = _oracle(im, q, r16, r8, b, mode)
        n = want["split"].size
        assert np.array_equal(recs[i], want["recon"]), i
        assert np.array_equal(split[k:k + n].astype(bool), want["split"].ravel()), i
        assert int(sse[i]) == want["sse"], i
        k += n


def test_mixed_1080p_frame(tx):
    img = synth.ar1_image(4244, 1088, 1920, 0.95, 8)
    recs, split, sse = _run(tx, [img], [(16.0, 16, 4, "auto")], [8])
    want = _oracle(img, 16.0, 16, 4, 8, "auto")
    assert np.array_equal(split.astype(bool), want["split"].ravel())
    assert np.array_equal(recs[0], want["recon"])
    assert int(sse[0]) == want["sse"]


def test_mixed_rejects_bad_arguments(tx):
    import torch

    t = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    d = tx.image(t)
    for qp in [(16.0, 0, 4, 0), (16.0, 16, 65, 0), (16.0, 16, 4, 3), (float("nan"), 16, 4, 0)]:
        with pytest.raises(tx.Tx16Error):
            tx.tx16_codec_mixed([d], None, [qp])
    with pytest.raises(tx.Tx16Error):
        tx.tx16_codec_mixed([tx.image(torch.zeros((20, 32), dtype=torch.uint8, device="cuda"))], None,
                            [(16.0, 16, 4, 0)])
