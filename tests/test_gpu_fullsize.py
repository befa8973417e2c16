"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times (one call over the whole batch), on sampled outputs the
oracle computes block by block, plus properties checked on every output.

  * 256 frames of 1920 x 1088 uint8 (the video model: one AR(1) field, rho
    0.95, cropped along a 2-pixel random walk), q = 16 and r in {4, 16, 32,
    256}: one tx16_codec_batch call (the kernel of each zonal class as timed),
    3000 random blocks and every tile-boundary block of the first and last
    frames against the oracle's binary32 decision path, bit-exact; every
    frame's squared error against the GPU's own reconstruction, exact.
  * 64 images of 2048 x 2048 uint8, forward only: 4000 random blocks and the
    first and last block of every image against the direct int64 product,
    bit-exact.  The forward path is data-independent arithmetic, so uniform
    random samples stand in for the AR(1) fields here.
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


@pytest.mark.parametrize("r", [16, 4, 32, 256])
def test_headline_workload_full_size(tx, frames, r):
    import torch

    n, H, W = frames.shape
    q = 16.0
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
