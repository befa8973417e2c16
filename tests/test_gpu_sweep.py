"""Zonal sweep (the paper's Fig. 2 experiment) against the oracle: one
forward per block, exact reconstruction for every r of the list."""
import numpy as np
import pytest

from helpers import to_dev
from oracle import tx16_oracle as O
from paper_1606_07414_gb300 import synth

pytestmark = pytest.mark.gpu

R_LIST = [1, 2, 4, 8, 16, 32, 64, 100, 128, 150, 256]


@pytest.fixture(scope="module")
def tx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1606_07414_gb300 import build, tx16

    build.build()
    tx16.load()
    return tx16


def test_sweep_matches_oracle_per_r(tx):
    import torch

    imgs = [synth.ar1_image(1, 512, 512, 0.95), synth.ar1_image(2, 80, 272, 0.9),
            synth.ar1_image(3, 48, 64, 0.95, bits=10)]
    keep = [to_dev(im) for im in imgs]  # descriptors hold raw pointers: keep tensors alive
    devs = [tx.image(t, 10 if im.dtype == np.uint16 else 8) for t, im in zip(keep, imgs)]
    sse = torch.full((len(imgs) * len(R_LIST),), 7, dtype=torch.int64, device="cuda")
    tx.tx16_zonal_sweep(devs, R_LIST, sse)
    got = sse.cpu().numpy().reshape(len(imgs), len(R_LIST))
    for i, im in enumerate(imgs):
        bits = 10 if im.dtype == np.uint16 else 8
        for j, r in enumerate(R_LIST):
            assert got[i, j] == O.codec_image(im, None, r, bits)["sse"], (i, r)
    assert np.all(got[:, -1] == 0)  # r = 256 reconstructs exactly


def test_sweep_equals_one_codec_call_per_r(tx):
    import torch

    img = to_dev(synth.ar1_image(9, 1088, 1920, 0.95))
    sse = torch.zeros(4, dtype=torch.int64, device="cuda")
    tx.tx16_zonal_sweep([img], [3, 16, 45, 150], sse)
    for j, r in enumerate([3, 16, 45, 150]):
        s1 = torch.zeros(1, dtype=torch.int64, device="cuda")
        tx.tx16_codec_batch([img], None, [(None, r)], sse=s1)
        assert int(s1.item()) == int(sse[j].item())


def test_sweep_extreme_planes_all_depths(tx):
    """Planes of extreme samples (checkerboards, stripes and a step of 0 and
    the peak) at 8, 10 and 12 bits: large per-row errors in the warp sums and
    reconstructions clipped at both ends, exact against the oracle for every r."""
    import torch

    ii, jj = np.indices((48, 64))
    imgs, bitss = [], []
    for bits in (8, 10, 12):
        peak = (1 << bits) - 1
        dt = np.uint8 if bits == 8 else np.uint16
        for pat in (((ii + jj) % 2) * peak, ((jj // 3) % 2) * peak, (jj >= 21) * peak):
            imgs.append(pat.astype(dt))
            bitss.append(bits)
    keep = [to_dev(im) for im in imgs]
    devs = [tx.image(t, b) for t, b in zip(keep, bitss)]
    sse = torch.full((len(imgs) * len(R_LIST),), 7, dtype=torch.int64, device="cuda")
    tx.tx16_zonal_sweep(devs, R_LIST, sse)
    got = sse.cpu().numpy().reshape(len(imgs), len(R_LIST))
    for i, (im, bits) in enumerate(zip(imgs, bitss)):
        for j, r in enumerate(R_LIST):
            assert got[i, j] == O.codec_image(im, None, r, bits)["sse"], (i, bits, r)
