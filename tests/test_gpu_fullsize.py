"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times (one call over the whole batch), on sampled outputs the
oracle computes block by block, plus properties checked on every output.

  * 256 frames of 1920 x 1088 uint8 (the video model: one AR(1) field, rho
    0.95, cropped along a 2-pixel random walk), the bench's sweep points (q in
    {8, 16, 32}, r in {4, 16, 32, 64, 128, 256}): one tx16_codec_batch call
    (the kernel of each zonal class as timed), 3000 random blocks and every
    tile-boundary block of the first and last frames against the oracle's
    binary32 decision path, bit-exact; every frame's squared error against the
    GPU's own reconstruction, exact; the PSNR of two full frames within
    1e-3 dB of the float64 definition.
  * 64 images of 2048 x 2048 uint8, forward only: 4000 random blocks and the
    first and last block of every image against the direct int64 product,
    bit-exact.  The forward path is data-independent arithmetic, so uniform
    random samples stand in for the AR(1) fields here.
  * 2000 uneven images through one plan, and the serving mix's request shapes
    through the server (below).
"""
import numpy as np
import pytest

from helpers import oracle_blocks
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


@pytest.fixture(scope="module")
def frames():
    return synth.video_frames(2016, 256, 1088, 1920, rho=0.95)


def _blocks(plane, picks, nbx):
    return np.stack([plane[(b // nbx) * 16:(b // nbx) * 16 + 16, (b % nbx) * 16:(b % nbx) * 16 + 16] for b in picks])


@pytest.mark.parametrize("q,r", [(16.0, 16), (16.0, 4), (16.0, 32), (16.0, 256), (8.0, 16), (32.0, 16),
                                 (16.0, 64), (8.0, 64), (32.0, 128)])
def test_headline_workload_full_size(tx, frames, q, r):
    """One call over the 256 frames of the bench's sweep points (every zonal
    class, q in {8, 16, 32}); sampled blocks bit-exact against the oracle's
    binary32 decision path, every frame's squared error exact, and the PSNR
    of the first and last full frames within 1e-3 dB of the float64
    definition (the paper's arithmetic, Sec. 3.1)."""
    import torch

    n, H, W = frames.shape
    d_in = torch.from_numpy(frames).cuda()
    d_out = torch.zeros_like(d_in)
    sse = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    tx.tx16_codec_batch([tx.image(d_in[i]) for i in range(n)], [tx.image(d_out[i]) for i in range(n)],
                        [(q, r)] * n, sse=sse)
    torch.cuda.synchronize()
    rec = d_out.cpu().numpy()
    s = sse.cpu().numpy()
    for i in range(n):  # every frame's squared error, exact
        assert int(s[i]) == O.sse(frames[i], rec[i]), i
    nbx, nb = W // 16, (H // 16) * (W // 16)
    rng = np.random.default_rng(1000 + r)
    picks = {}
    for g in rng.integers(0, n * nb, 3000).tolist():
        picks.setdefault(g // nb, set()).add(g % nb)
    edges = {b for t in range(0, nb, 32) for b in (t, t + 31) if b < nb} | {nb - 1}
    picks.setdefault(0, set()).update(edges)
    picks.setdefault(n - 1, set()).update(edges)
    X = np.concatenate([_blocks(frames[i], sorted(p), nbx) for i, p in sorted(picks.items())])
    got = np.concatenate([_blocks(rec[i], sorted(p), nbx) for i, p in sorted(picks.items())])
    ref = oracle_blocks(X.astype(np.int64), q, r, 8)
    assert np.array_equal(got, ref["recon"])
    psnr = tx.tx16_psnr([int(s[0]), int(s[n - 1])], [tx.image(d_in[0]), tx.image(d_in[n - 1])])
    for got_db, i in zip(psnr, (0, n - 1)):
        want = O.codec_image(frames[i], q, r, 8, "fp64")["psnr"]
        assert abs(got_db - want) <= 1e-3, (i, got_db, want)


def test_forward_full_size(tx):
    import torch

    n, S = 64, 2048
    rng = np.random.default_rng(64)
    imgs = rng.integers(0, 256, (n, S, S), dtype=np.uint8)
    d_in = torch.from_numpy(imgs).cuda()
    nb = (S // 16) ** 2
    coeffs = torch.empty((n * nb * 256,), dtype=torch.int32, device="cuda")
    tx.tx16_forward([tx.image(d_in[i]) for i in range(n)], coeffs)
    torch.cuda.synchronize()
    nbx = S // 16
    g = np.unique(np.concatenate([rng.integers(0, n * nb, 4000), np.arange(n) * nb, np.arange(1, n + 1) * nb - 1]))
    idx = torch.from_numpy(g).cuda()
    got = coeffs.view(n * nb, 256)[idx].cpu().numpy().reshape(-1, 16, 16)
    X = np.stack([_blocks(imgs[b // nb], [b % nb], nbx)[0] for b in g])
    assert np.array_equal(got, O.forward_direct(X.astype(np.int64)))


def test_uneven_batch_full_size(tx):
    """2000 images with sides drawn independently from the multiples of 16 in
    [64, 4096] (3.3e7 blocks), zonal r in {8, 32, 128}, q = 16, as crops of
    two 4096 x 4096 AR(1) fields: one plan, replayed as a CUDA graph.  Every
    image's squared error equals the separate unfused SSE kernel's over the
    same reconstruction; 3000 sampled blocks match the oracle bit for bit."""
    import torch

    n, side = 2000, 4096
    Hs, Ws = synth.uneven_sizes(2016 + 9, n)
    rs = synth.choice(2016 + 10, n, [8, 32, 128])
    u = synth.uniforms(2016 + 11, 2 * n)
    fields = [torch.from_numpy(synth.ar1_image(2016 + 700 + i, side, side, rho)).cuda()
              for i, rho in enumerate((0.9, 0.97))]
    ins, outs, qps = [], [], []
    for i in range(n):
        H, W = int(Hs[i]), int(Ws[i])
        y = min(int(u[2 * i] * (side - H + 1)), side - H)
        x = 16 * min(int(u[2 * i + 1] * ((side - W) // 16 + 1)), (side - W) // 16)
        ins.append(fields[i % 2][y:y + H, x:x + W])
        outs.append(torch.empty((H, W), dtype=torch.uint8, device="cuda"))
        qps.append((16.0, int(rs[i])))
    plan = tx.Plan(ins, outs, qps)
    sse = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    plan.run_graph(sse=sse)
    sse2 = torch.zeros(n, dtype=torch.int64, device="cuda")
    tx.tx16_sse(ins, outs, sse2)
    torch.cuda.synchronize()
    assert torch.equal(sse, sse2)
    rng = np.random.default_rng(2000)
    by_r = {}
    for i in rng.integers(0, n, 3000).tolist():
        nbx = int(Ws[i]) // 16
        b = int(rng.integers(0, (int(Hs[i]) // 16) * nbx))
        y, x = (b // nbx) * 16, (b % nbx) * 16
        X = ins[i][y:y + 16, x:x + 16].cpu().numpy()
        R = outs[i][y:y + 16, x:x + 16].cpu().numpy()
        by_r.setdefault(int(rs[i]), []).append((X, R))
    for r, pairs in by_r.items():
        X = np.stack([p[0] for p in pairs]).astype(np.int64)
        got = np.stack([p[1] for p in pairs])
        assert np.array_equal(got, oracle_blocks(X, 16.0, r, 8)["recon"]), r
    plan.close()


def test_serving_request_shapes_full_size(tx):
    """The serving mix's request shapes at full size (256 x 256 and
    1920 x 1088 uint8, 3840 x 2160 10-bit in uint16), each with its own q and
    r, submitted together so that they are admitted and coded in groups:
    every result equals a direct tx16_codec_batch call on the same image, bit
    for bit, with the same PSNR, and sampled blocks match the oracle."""
    import torch

    kinds = synth.choice(5, 30, [0, 0, 0, 0, 0, 0, 1, 1, 1, 2])
    qs = synth.choice(6, 30, [8.0, 16.0, 32.0])
    rs = synth.choice(7, 30, [4, 16, 64, 256])
    reqs = []
    for i in range(30):
        if kinds[i] == 0:
            img, bits = synth.ar1_image(300 + i, 256, 256, 0.95), 8
        elif kinds[i] == 1:
            img, bits = synth.ar1_image(300 + i, 1088, 1920, 0.95), 8
        else:
            img, bits = synth.ar1_image(300 + i, 2160, 3840, 0.95, bits=10), 10
        reqs.append((img, bits, float(qs[i]), int(rs[i])))
    srv = tx.Server({"device_pool_mb": 2048, "streams": 3, "max_batch": 64})
    outs = [np.zeros_like(img) for img, _, _, _ in reqs]
    tickets = [srv.submit(img, q, r, out=o, bits=bits) for (img, bits, q, r), o in zip(reqs, outs)]
    psnrs = [srv.wait(t)[0] for t in tickets]
    srv.close()
    rng = np.random.default_rng(30)
    for (img, bits, q, r), o, p in zip(reqs, outs, psnrs):
        d = torch.from_numpy(img.view(np.int16) if bits > 8 else img).cuda()
        rec = torch.empty_like(d)
        s = torch.zeros(1, dtype=torch.int64, device="cuda")
        tx.tx16_codec_batch([tx.image(d, bits)], [tx.image(rec, bits)], [(q, r)], sse=s)
        torch.cuda.synchronize()
        assert np.array_equal(o, rec.cpu().numpy().view(img.dtype))
        assert p == tx.tx16_psnr([int(s.item())], [tx.image(d, bits)])[0]
        H, W = img.shape
        nbx = W // 16
        picks = rng.integers(0, (H // 16) * nbx, 40)
        X = _blocks(img, picks, nbx).astype(np.int64)
        assert np.array_equal(_blocks(o, picks, nbx), oracle_blocks(X, q, r, bits)["recon"])
