"""Serving loop: results are the same alone and in a mix of concurrent
requests, admission and errors behave (no GPU fault involved: failures are
made on the host), statistics are sane."""
import numpy as np
import pytest

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


def _mix(seed, n):
    """Request mix: small 8-bit, frame-sized 8-bit and 10-bit planes."""
    reqs = []
    kinds = synth.choice(seed, n, [0, 0, 0, 1, 1, 2])
    qs = synth.choice(seed + 1, n, [8.0, 16.0, 32.0, None])
    rs = synth.choice(seed + 2, n, [4, 16, 64, 256])
    for i in range(n):
        if kinds[i] == 0:
            img, bits = synth.ar1_image(seed * 7 + i, 64, 96, 0.95), 8
        elif kinds[i] == 1:
            img, bits = synth.ar1_image(seed * 7 + i, 272, 480, 0.95), 8
        else:
            img, bits = synth.ar1_image(seed * 7 + i, 144, 256, 0.95, bits=10), 10
        q = None if qs[i] is None else float(qs[i])
        reqs.append((img, bits, q, int(rs[i])))
    return reqs


def test_same_result_alone_and_in_the_mix(tx):
    srv = tx.Server({"device_pool_mb": 256, "streams": 3, "max_batch": 64})
    probe = synth.ar1_image(4242, 272, 480, 0.95)
    out_alone = np.zeros_like(probe)
    t = srv.submit(probe, 16.0, 64, out=out_alone)
    psnr_alone, _ = srv.wait(t)
    ref = O.codec_image(probe, 16.0, 64, 8, "fp32")
    assert np.array_equal(out_alone, ref["recon"])
    assert psnr_alone == pytest.approx(ref["psnr"], abs=1e-9)

    reqs = _mix(17, 300)
    outs, tickets = [], []
    out_mix = np.zeros_like(probe)
    for i, (img, bits, q, r) in enumerate(reqs):
        o = np.zeros_like(img)
        outs.append(o)
        tickets.append(srv.submit(img, q, r, out=o, bits=bits))
        if i == 150:
            tp = srv.submit(probe, 16.0, 64, out=out_mix)
    psnrs = [srv.wait(t)[0] for t in tickets]
    psnr_mix, _ = srv.wait(tp)
    assert np.array_equal(out_mix, out_alone) and psnr_mix == psnr_alone
    # every request of the mix against the oracle (binary32 decision path)
    for (img, bits, q, r), o, p in zip(reqs, outs, psnrs):
        ref = O.codec_image(img, q, r, bits, "fp32" if q else "fp64")
        assert np.array_equal(o, ref["recon"])
        assert (p == ref["psnr"]) if not np.isfinite(ref["psnr"]) else p == pytest.approx(ref["psnr"], abs=1e-9)
    st = srv.stats()
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["p999_us"] and st["mblocks_per_s"] > 0
    srv.close()


def test_admission_and_errors_made_on_the_host(tx):
    srv = tx.Server({"device_pool_mb": 1, "streams": 1, "max_batch": 4, "max_queue": 2})
    small = synth.ar1_image(1, 64, 64, 0.9)
    with pytest.raises(tx.Tx16Error) as e:  # shape not a multiple of 16
        srv.submit(np.zeros((60, 64), np.uint8), 16.0, 16)
    assert e.value.status == tx.TX16_EINVAL
    with pytest.raises(tx.Tx16Error) as e:  # r out of range
        srv.submit(small, 16.0, 0)
    assert e.value.status == tx.TX16_EINVAL
    with pytest.raises(tx.Tx16Error) as e:  # larger than the whole arena: never admissible
        srv.submit(np.zeros((1024, 1024), np.uint8), 16.0, 16)
    assert e.value.status == tx.TX16_ENOMEM
    srv.pause(True)  # admission held: the queue fills deterministically
    t1 = srv.submit(small, 16.0, 16)
    t2 = srv.submit(small, 8.0, 4)
    with pytest.raises(tx.Tx16Error) as e:
        srv.submit(small, 16.0, 16)
    assert e.value.status == tx.TX16_EBUSY
    with pytest.raises(tx.Tx16Error) as e:  # nothing admitted while paused: bounded wait ends
        srv.wait(t1, timeout_ms=50)
    assert e.value.status == tx.TX16_ETIMEOUT
    srv.pause(False)
    p1, _ = srv.wait(t1)
    p2, _ = srv.wait(t2)
    assert p1 == pytest.approx(O.codec_image(small, 16.0, 16, 8, "fp32")["psnr"], abs=1e-9)
    assert p2 == pytest.approx(O.codec_image(small, 8.0, 4, 8, "fp32")["psnr"], abs=1e-9)
    with pytest.raises(tx.Tx16Error) as e:  # a released ticket is unknown
        srv.wait(t1)
    assert e.value.status == tx.TX16_EINVAL
    # the arena holds about one request at a time: many still complete in order
    ts = []
    for i in range(12):
        ts.append(srv.submit(small, 16.0, 16))
        if len(ts) >= 2:
            srv.wait(ts.pop(0))
    for t in ts:
        srv.wait(t)
    # destroy with work queued: it drains
    srv.pause(True)
    srv.submit(small, 16.0, 16)
    srv.close()


@pytest.mark.parametrize("spin_us", [0, 20000])
def test_polling_window_does_not_change_results(tx, spin_us):
    """spin_us = 0 blocks at once (completion learnt from the slot callbacks);
    a long window keeps the worker polling slot events throughout."""
    srv = tx.Server({"device_pool_mb": 64, "streams": 2, "max_batch": 8, "spin_us": spin_us})
    reqs = _mix(23, 40)
    outs, tickets = [], []
    for img, bits, q, r in reqs:
        o = np.zeros_like(img)
        outs.append(o)
        tickets.append(srv.submit(img, q, r, out=o, bits=bits))
    for (img, bits, q, r), o, t in zip(reqs, outs, tickets):
        p, lat = srv.wait(t)
        ref = O.codec_image(img, q, r, bits, "fp32" if q else "fp64")
        assert np.array_equal(o, ref["recon"]) and lat > 0
    srv.close()


def test_bad_polling_window_is_rejected(tx):
    for bad in (-1, 2e6, float("nan")):
        with pytest.raises(tx.Tx16Error) as e:
            tx.Server({"spin_us": bad})
        assert e.value.status == tx.TX16_EINVAL


@pytest.mark.parametrize("band_mb", [0.0, 0.01, 0.05])
def test_bands_do_not_change_results(tx, band_mb):
    """Planes above band_mb are copied in, coded and copied out in bands of
    whole block rows (up to 8; the band count of a group differs from request
    to request): samples and PSNR stay those of the oracle, the per-band
    squared errors summing to the plane's."""
    srv = tx.Server({"device_pool_mb": 128, "streams": 3, "max_batch": 16, "band_mb": band_mb})
    reqs = _mix(31, 60)
    outs, tickets = [], []
    for img, bits, q, r in reqs:
        o = np.zeros_like(img)
        outs.append(o)
        tickets.append(srv.submit(img, q, r, out=o, bits=bits))
    for (img, bits, q, r), o, t in zip(reqs, outs, tickets):
        p, lat = srv.wait(t)
        ref = O.codec_image(img, q, r, bits, "fp32" if q else "fp64")
        assert np.array_equal(o, ref["recon"])
        assert (p == ref["psnr"]) if not np.isfinite(ref["psnr"]) else p == pytest.approx(ref["psnr"], abs=1e-9)
    srv.close()


def test_bad_band_size_is_rejected(tx):
    for bad in (-1, 1e9, float("nan")):
        with pytest.raises(tx.Tx16Error) as e:
            tx.Server({"band_mb": bad})
        assert e.value.status == tx.TX16_EINVAL
