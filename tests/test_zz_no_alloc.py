"""tx16_codec_batch_static: the codec for callers that cannot allocate device
memory where they run it (their card belongs to another allocator's pool, an
allocation would synchronise a latency-critical loop, or their memory budget
is fixed at start-up).  Its work list lives in a fixed array inside the
library, so consecutive calls share that array.

Checked through the C-ABI against the existing entry points of the same
work-list kernel (a plan, which allocates its list) and tx16_codec_batch,
bit for bit, on two calls in a row with different batches.  This file is
collected last so that a run stopping at the first failure has run every
other test first.
"""
import ctypes

import numpy as np
import pytest

from helpers import empty_like_img, to_dev
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


def _batch(seed, n, lo, hi, qs, rs):
    Hs, Ws = synth.uneven_sizes(seed, n, lo, hi)
    imgs = [synth.ar1_image(seed * 1000 + i, int(Hs[i]), int(Ws[i]), 0.9) for i in range(n)]
    qp = [(qs[i % len(qs)], rs[i % len(rs)]) for i in range(n)]
    return imgs, qp


def _static_call(tx, ins, outs, qp, sse, levels):
    """Call the entry point through the C-ABI directly."""
    import torch

    lib = tx.load()
    n = len(ins)
    in_arr = (tx.tx16_image * n)(*[tx.image(t) for t in ins])
    out_arr = (tx.tx16_image * n)(*[tx.image(t) for t in outs])
    qp_arr = (tx.tx16_qparams * n)(*[tx.tx16_qparams(0.0 if q is None else q, r) for q, r in qp])
    st = lib.tx16_codec_batch_static(in_arr, out_arr, n, qp_arr, ctypes.c_void_p(sse.data_ptr()),
                                     ctypes.c_void_p(levels.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == tx.TX16_OK, tx.status_str(st)


def test_static_entry_point_matches_allocating_ones_twice(tx):
    import torch

    batches = [_batch(21, 30, 16, 512, [16.0, None, 8.0], [16, 64, 8, 256]),
               _batch(22, 17, 32, 768, [32.0, 5.3], [4, 128, 32])]
    for imgs, qp in batches:  # two calls in a row: the shared array must not leak state
        ins = [to_dev(im) for im in imgs]
        nb = sum((im.shape[0] // 16) * (im.shape[1] // 16) for im in imgs)
        out_s = [empty_like_img(*im.shape, 8) for im in imgs]
        out_p = [empty_like_img(*im.shape, 8) for im in imgs]
        out_b = [empty_like_img(*im.shape, 8) for im in imgs]
        lev_s = torch.full((nb * 256,), 0x7EADBEEF, dtype=torch.int32, device="cuda")
        lev_p = torch.zeros_like(lev_s)
        sse_s = torch.full((len(imgs),), 99, dtype=torch.int64, device="cuda")
        sse_p = torch.zeros_like(sse_s)
        sse_b = torch.zeros_like(sse_s)
        _static_call(tx, ins, out_s, qp, sse_s, lev_s)
        plan = tx.Plan(ins, out_p, qp, bits=8)
        plan.run(sse=sse_p, levels=lev_p)
        tx.tx16_codec_batch(ins, out_b, qp, sse=sse_b, bits=8)
        torch.cuda.synchronize()
        for a, b, c in zip(out_s, out_p, out_b):
            assert torch.equal(a, b) and torch.equal(a, c)
        assert torch.equal(sse_s, sse_p) and torch.equal(sse_s, sse_b)
        assert torch.equal(lev_s, lev_p)
        plan.close()


def test_static_entry_point_rejects_batches_beyond_its_array(tx):
    import torch

    img = to_dev(synth.ar1_image(3, 16, 16, 0.9))
    out = empty_like_img(16, 16, 8)
    n = tx.TX16_STATIC_MAX_IMAGES + 1
    with pytest.raises(tx.Tx16Error) as e:
        tx.tx16_codec_batch_static([img] * n, [out] * n, [(16.0, 16)] * n)
    assert e.value.status == tx.TX16_EINVAL
    # exactly at the limit is accepted
    n = tx.TX16_STATIC_MAX_IMAGES
    sse = torch.zeros(n, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch_static([img] * n, [out] * n, [(16.0, 16)] * n, sse=sse)
    torch.cuda.synchronize()
    assert np.all(sse.cpu().numpy() == sse[0].item())
