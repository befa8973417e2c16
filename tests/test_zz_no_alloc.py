"""tx16_codec_batch_static: the codec for callers that cannot allocate device
memory where they run it (their card belongs to another allocator's pool, an
allocation would synchronise a latency-critical loop, or their memory budget
is fixed at start-up).  Its work list lives in a fixed array inside the
library, so consecutive calls share that array.

Checked through the C-ABI against the existing entry points of the same
work-list kernel (a plan, which allocates its list) and tx16_codec_batch,
bit for bit, on two calls in a row with different batches, 8-bit and 10-bit;
that a call changes neither the device's free memory nor torch's allocation
count; and, at the size limit, against the oracle.  This file is collected
last so that a run stopping at the first failure has run every other test
first.
"""
import ctypes

import numpy as np
import pytest

from helpers import empty_like_img, to_dev
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


def _batch(seed, n, lo, hi, qs, rs, bits=None):
    """n AR(1) images with uneven sides; bits[i] per image (8 by default)."""
    Hs, Ws = synth.uneven_sizes(seed, n, lo, hi)
    bits = bits or [8] * n
    imgs = [synth.ar1_image(seed * 1000 + i, int(Hs[i]), int(Ws[i]), 0.9, bits=bits[i]) for i in range(n)]
    qp = [(qs[i % len(qs)], rs[i % len(rs)]) for i in range(n)]
    return imgs, qp, bits


def _descs(tx, ts, bits):
    return [tx.image(t, b) for t, b in zip(ts, bits)]


def _static_call(tx, ins, outs, qp, sse, levels):
    """Call the entry point through the C-ABI directly (ins/outs: descriptors)."""
    import torch

    lib = tx.load()
    n = len(ins)
    in_arr = (tx.tx16_image * n)(*ins)
    out_arr = (tx.tx16_image * n)(*outs)
    qp_arr = (tx.tx16_qparams * n)(*[tx.tx16_qparams(0.0 if q is None else q, r) for q, r in qp])
    st = lib.tx16_codec_batch_static(in_arr, out_arr, n, qp_arr, ctypes.c_void_p(sse.data_ptr()),
                                     ctypes.c_void_p(0 if levels is None else levels.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == tx.TX16_OK, tx.status_str(st)


def _compare_with_allocating_calls(tx, imgs, qp, bits, with_levels):
    import torch

    ins = [to_dev(im) for im in imgs]
    din = _descs(tx, ins, bits)
    nb = sum((im.shape[0] // 16) * (im.shape[1] // 16) for im in imgs)
    out_s = [empty_like_img(*im.shape, b) for im, b in zip(imgs, bits)]
    out_p = [empty_like_img(*im.shape, b) for im, b in zip(imgs, bits)]
    out_b = [empty_like_img(*im.shape, b) for im, b in zip(imgs, bits)]
    lev_s = lev_p = None
    if with_levels:
        lev_s = torch.full((nb * 256,), 0x7EADBEEF, dtype=torch.int32, device="cuda")
        lev_p = torch.zeros_like(lev_s)
    sse_s = torch.full((len(imgs),), 99, dtype=torch.int64, device="cuda")
    sse_p = torch.zeros_like(sse_s)
    sse_b = torch.zeros_like(sse_s)
    _static_call(tx, din, _descs(tx, out_s, bits), qp, sse_s, lev_s)
    plan = tx.Plan(din, _descs(tx, out_p, bits), qp)
    plan.run(sse=sse_p, levels=lev_p)
    tx.tx16_codec_batch(din, _descs(tx, out_b, bits), qp, sse=sse_b)
    torch.cuda.synchronize()
    for a, b, c in zip(out_s, out_p, out_b):
        assert torch.equal(a, b) and torch.equal(a, c)
    assert torch.equal(sse_s, sse_p) and torch.equal(sse_s, sse_b)
    if with_levels:
        assert torch.equal(lev_s, lev_p)
    plan.close()
    return out_s, sse_s


def test_static_entry_point_matches_allocating_ones_twice(tx):
    batches = [_batch(21, 30, 16, 512, [16.0, None, 8.0], [16, 64, 8, 256]),
               _batch(22, 17, 32, 768, [32.0, 5.3], [4, 128, 32])]
    for imgs, qp, bits in batches:  # two calls in a row: the shared array must not leak state
        _compare_with_allocating_calls(tx, imgs, qp, bits, with_levels=True)


def test_static_entry_point_mixed_8_and_10_bit_twice(tx):
    """9..12-bit planes take the general kernel, one launch per image with its
    own squared-error slot; 8-bit planes the work-list kernel, in one call."""
    for seed in (23, 24):
        bits = [8, 10, 8, 12, 10, 8, 9]
        imgs, qp, bits = _batch(seed, len(bits), 16, 320, [16.0, 40.0, None], [16, 64, 200], bits)
        outs, sse = _compare_with_allocating_calls(tx, imgs, qp, bits, with_levels=False)
        for im, o, s, b, (q, r) in zip(imgs, outs, sse.cpu().tolist(), bits, qp):
            ref = O.codec_image(im, q, r, b, "fp32")
            got = o.cpu().numpy()
            got = got.view(np.uint16) if b > 8 else got
            assert np.array_equal(got, ref["recon"])
            assert s == ref["sse"]


def test_static_entry_point_allocates_nothing(tx):
    """After one warm-up call (which may load the kernels' code), a call
    leaves the device's free memory and torch's allocation count unchanged."""
    import torch

    imgs, qp, bits = _batch(25, 12, 32, 640, [16.0, None], [16, 64, 256])
    ins = _descs(tx, [to_dev(im) for im in imgs], bits)
    outs = _descs(tx, [empty_like_img(*im.shape, 8) for im in imgs], bits)
    sse = torch.zeros(len(imgs), dtype=torch.int64, device="cuda")
    _static_call(tx, ins, outs, qp, sse, None)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        _static_call(tx, ins, outs, qp, sse, None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0


def test_static_entry_point_rejects_batches_beyond_its_array(tx):
    import torch

    im = synth.ar1_image(3, 16, 16, 0.9)
    img = to_dev(im)
    out = empty_like_img(16, 16, 8)
    n = tx.TX16_STATIC_MAX_IMAGES + 1
    with pytest.raises(tx.Tx16Error) as e:
        tx.tx16_codec_batch_static([img] * n, [out] * n, [(16.0, 16)] * n)
    assert e.value.status == tx.TX16_EINVAL
    # exactly at the limit is accepted, and every image's error is the oracle's
    n = tx.TX16_STATIC_MAX_IMAGES
    sse = torch.zeros(n, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch_static([img] * n, [out] * n, [(16.0, 16)] * n, sse=sse)
    torch.cuda.synchronize()
    ref = O.codec_image(im, 16.0, 16, 8, "fp32")
    assert np.all(sse.cpu().numpy() == ref["sse"])
    assert np.array_equal(out.cpu().numpy(), ref["recon"])
