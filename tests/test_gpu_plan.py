"""GPU parity of batch plans (device work list, persistent launches, CUDA
graph replay, autotuned schedules) against the oracle and against
tx16_codec_batch on the same images."""
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


def _batch(seed, n, lo=16, hi=400, bits_mix=False):
    Hs, Ws = synth.uneven_sizes(seed, n, lo, hi)
    rs = synth.choice(seed + 1, n, [8, 32, 128])
    qs = synth.choice(seed + 2, n, [None, 8.0, 16.0, 32.0]) if not bits_mix else [16.0] * n
    imgs = []
    for i in range(n):
        b = 10 if (bits_mix and i % 3 == 0) else 8
        imgs.append(synth.ar1_image(seed * 100 + i, int(Hs[i]), int(Ws[i]), 0.8 + 0.18 * (i % 7) / 6, b))
    return imgs, [(None if q is None else float(q), int(r)) for q, r in zip(qs, rs)]


@pytest.mark.parametrize("graph", [False, True])
def test_plan_matches_oracle_uneven_batch(tx, graph):
    import torch

    imgs, qp = _batch(5, 24)
    ins = [to_dev(im) for im in imgs]
    outs = [empty_like_img(*im.shape, 8) for im in imgs]
    plan = tx.Plan(ins, outs, qp, bits=8)
    nb = sum((im.shape[0] // 16) * (im.shape[1] // 16) for im in imgs)
    lev = torch.full((nb * 256,), 0x7EADBEEF, dtype=torch.int32, device="cuda")
    sse = torch.zeros(len(imgs), dtype=torch.int64, device="cuda")
    for _ in range(2):  # a second run must reset counters and SSE itself
        (plan.run_graph if graph else plan.run)(sse=sse, levels=lev)
    torch.cuda.synchronize()
    L = lev.cpu().numpy().reshape(nb, 16, 16)
    k = 0
    for i, im in enumerate(imgs):
        n = (im.shape[0] // 16) * (im.shape[1] // 16)
        q, r = qp[i]
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, 8)
        assert np.array_equal(L[k:k + n], ref["levels"]), i
        rec = from_dev(outs[i], 8)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i
        k += n
    assert len(plan.info()) >= 2  # several zone classes in this batch
    plan.close()


def test_plan_equals_codec_batch_and_survives_autotune(tx, tmp_path):
    import torch

    imgs, qp = _batch(9, 40, 16, 640)
    ins = [to_dev(im) for im in imgs]
    outs1 = [empty_like_img(*im.shape, 8) for im in imgs]
    outs2 = [empty_like_img(*im.shape, 8) for im in imgs]
    s1 = torch.zeros(len(imgs), dtype=torch.int64, device="cuda")
    s2 = torch.zeros(len(imgs), dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch(ins, outs1, qp, sse=s1, bits=8)
    plan = tx.Plan(ins, outs2, qp, bits=8)
    cache = str(tmp_path / "tune.txt")
    plan.autotune(cache)
    plan.run_graph(sse=s2)
    torch.cuda.synchronize()
    for a, b in zip(outs1, outs2):
        assert torch.equal(a, b)
    assert torch.equal(s1, s2)
    # a second plan reads the cached schedules
    plan2 = tx.Plan(ins, outs2, qp, bits=8)
    plan2.autotune(cache)
    assert [r["chunk"] for r in plan2.info()] == [r["chunk"] for r in plan.info()]
    plan.close()
    plan2.close()


def test_plan_mixed_depths_and_tiny_steps(tx):
    """16-bit planes and steps below the fused kernel's range take the
    general kernel inside the same plan."""
    import torch

    imgs, qp = _batch(13, 9, 16, 160, bits_mix=True)
    qp[1] = (2.0 ** -10, 256)
    tens_in = [to_dev(im) for im in imgs]
    ins = [tx.image(t, 10 if im.dtype == np.uint16 else 8) for t, im in zip(tens_in, imgs)]
    outs_t = [empty_like_img(*im.shape, 10 if im.dtype == np.uint16 else 8) for im in imgs]
    outs = [tx.image(t, 10 if im.dtype == np.uint16 else 8) for t, im in zip(outs_t, imgs)]
    sse = torch.zeros(len(imgs), dtype=torch.int64, device="cuda")
    plan = tx.Plan(ins, outs, qp)
    plan.run(sse=sse)
    torch.cuda.synchronize()
    for i, im in enumerate(imgs):
        b = 10 if im.dtype == np.uint16 else 8
        q, r = qp[i]
        ref = oracle_blocks(O.image_to_blocks(im.astype(np.int64)), q, r, b)
        rec = from_dev(outs_t[i], b)
        assert np.array_equal(O.image_to_blocks(rec.astype(np.int64)), ref["recon"]), i
        assert int(sse[i].item()) == O.sse(im, rec), i
    plan.close()


def test_every_compiled_configuration_gives_identical_results(tx):
    """Each fused group has two mappings of blocks to lanes: the pair kernel
    (variant -1) and the one-block-per-thread kernel in several compiled
    configurations (warps per CTA, parked column pairs, input stages).
    Pinned one by one, with different CTAs per SM and tiles per claim, every
    mapping and configuration writes the same samples and squared errors (and
    the first run matches the oracle)."""
    import torch

    Hs, Ws = synth.uneven_sizes(31, 36, 16, 720)
    rs = [4, 8, 16, 32, 64, 24, 48, 12]
    qs = [16.0, None, 8.0, 32.0]
    imgs = [synth.ar1_image(3100 + i, int(Hs[i]), int(Ws[i]), 0.85 + 0.02 * (i % 6), 8) for i in range(len(Hs))]
    qp = [(qs[i % 4], rs[i % 8]) for i in range(len(imgs))]
    ins = [to_dev(im) for im in imgs]
    outs = [empty_like_img(*im.shape, 8) for im in imgs]
    plan = tx.Plan(ins, outs, qp, bits=8)
    info = plan.info()
    tuned = [i for i, g in enumerate(info) if g["variant"] >= 0]
    assert {info[i]["zone"] for i in tuned} == {0, 1, 2, 3}  # r <= 8, 16, 32, 64 all present
    sse = torch.zeros(len(imgs), dtype=torch.int64, device="cuda")
    ref_out, ref_sse = None, None
    seen = set()
    for var in range(-1, 3):
        # chunk 0: no claims, a contiguous run of tiles per CTA (one block per thread)
        for ctas, chunk in ((0, 1), (1, 3)) + (((0, 0),) if var >= 0 else ()):
            for i in tuned:
                plan.set_schedule(i, var, ctas, chunk)
            for o in outs:
                o.zero_()
            plan.run(sse=sse)
            torch.cuda.synchronize()
            for i in tuned:
                g = plan.info()[i]
                assert g["variant"] == var and g["ctas_per_sm"] == ctas and g["chunk"] == chunk
                seen.add((g["zone"], var, g["warps_per_cta"], g["parked_pairs"], g["stages"]))
            got = [o.clone() for o in outs]
            if ref_out is None:
                ref_out, ref_sse = got, sse.clone()
                for im, o, (q, r) in zip(imgs, got, qp):
                    ref = O.codec_image(im, q, r, 8, "fp32")
                    assert np.array_equal(from_dev(o, 8), ref["recon"])
            else:
                for a, b in zip(ref_out, got):
                    assert torch.equal(a, b)
                assert torch.equal(ref_sse, sse)
    # the pair kernel and three distinct configurations per group, at least
    # one with two stages
    assert len(seen) == 16 and any(s[4] == 2 for s in seen)
    assert all(s[2:] == (0, 0, 0) for s in seen if s[1] == -1)
    with pytest.raises(tx.Tx16Error):
        plan.set_schedule(tuned[0], 3, 0, 1)
    plan.autotune(None)
    for i in tuned:
        assert -1 <= plan.info()[i]["variant"] < 3
    plan.close()
