"""GPU parity of tx16_ssim against the oracle's ``ssim_map`` / ``ssim``.

Tolerance, derived from the kernel's binary32 arithmetic (u = 2^-24,
g_n = n u / (1 - n u)).  With samples centred on c = 2^(bits-1)
(x' = x - c) and W[.] the window mean:

  * each local moment E is two 11-tap weighted sums of rounded products with
    rounded weights: |dE| <= g_30 W[|v|] (v = x', y', x'^2, y'^2, x'y');
  * s_x^2 = E x'^2 - (E x')^2 by one fma: |ds_x^2| <= (3 g_30 + u) W[x'^2];
    |ds_xy| <= (3 g_30 + 2u) sqrt(W[x'^2] W[y'^2]);
  * mu = E x' + c: |dmu| <= g_30 W[|x'|] + u |mu|;
  * N1 = 2 mu_x mu_y + C1, D1 = mu_x^2 + mu_y^2 + C1, N2 = 2 s_xy + C2,
    D2 = s_x^2 + s_y^2 + C2 (constants rounded to binary32), the index
    N1 N2 / (D1 D2): two rounded products and a fast division (at most 2 ulp,
    CUDA's documented bound for __fdividef in this range), 7u together;
  * |d index| <= |index| (dD1/D1 + dD2/D2 + 7u) + (dN1 |N2| + |N1| dN2) / (D1 D2),
    with the denominators reduced by their own error bounds; the test allows
    twice that per position;
  * the mean: the mean of the per-position bounds plus 72 u (binary32 partial
    sums of at most 64 indices per thread before the binary64 reduction).
"""
import numpy as np
import pytest

from oracle import tx16_oracle as O
from paper_1606_07414_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _gamma(n):
    return n * U / (1 - n * U)


@pytest.fixture(scope="module")
def tx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1606_07414_gb300 import build, tx16

    build.build()
    tx16.load()
    return tx16


def _bound(x, y, bits):
    """Per-position bound of |index_binary32 - index_binary64| (module doc)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    c = float(1 << (bits - 1))
    L = float((1 << bits) - 1)
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    w = O.ssim_window()
    xp, yp = x - c, y - c
    Ax, Ay = O.window_mean(np.abs(xp), w), O.window_mean(np.abs(yp), w)
    Qx, Qy = O.window_mean(xp * xp, w), O.window_mean(yp * yp, w)
    mx, my = O.window_mean(x, w), O.window_mean(y, w)
    sxx = O.window_mean(x * x, w) - mx * mx
    syy = O.window_mean(y * y, w) - my * my
    sxy = O.window_mean(x * y, w) - mx * my
    g = _gamma(30)
    dsxx = (3 * g + U) * Qx
    dsyy = (3 * g + U) * Qy
    dsxy = (3 * g + 2 * U) * np.sqrt(Qx * Qy)
    dmx = g * Ax + U * np.abs(mx)
    dmy = g * Ay + U * np.abs(my)
    N1 = 2 * mx * my + C1
    D1 = mx * mx + my * my + C1
    N2 = 2 * sxy + C2
    D2 = sxx + syy + C2
    dN1 = 2 * (np.abs(my) * dmx + np.abs(mx) * dmy + dmx * dmy) + U * (np.abs(N1) + C1)
    dD1 = 2 * (np.abs(mx) * dmx + np.abs(my) * dmy) + dmx ** 2 + dmy ** 2 + 2 * U * D1 + U * C1
    dN2 = 2 * dsxy + U * (np.abs(N2) + C2)
    dD2 = dsxx + dsyy + 2 * U * (np.abs(sxx) + np.abs(syy) + C2) + U * C2
    D1l, D2l = D1 - dD1, D2 - dD2
    assert np.all(D1l > 0) and np.all(D2l > 0)
    s = N1 * N2 / (D1 * D2)
    b = np.abs(s) * (dD1 / D1l + dD2 / D2l + 7 * U) + (dN1 * np.abs(N2) + np.abs(N1) * dN2) / (D1l * D2l)
    return 2 * b


def _dev(img, bits):
    """Upload with a 16-byte-multiple pitch (rows padded as needed)."""
    import torch

    H, W = img.shape
    per = 16 if bits == 8 else 8
    P = -(-W // per) * per
    dt = torch.uint8 if bits == 8 else torch.int16
    t = torch.zeros((H, P), dtype=dt, device="cuda")
    a = img.view(np.int16) if bits > 8 else img
    t[:, :W] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t, t[:, :W]


def _pair(seed, H, W, bits, q=16.0, r=16):
    """An AR(1) image and its reconstruction by the oracle's codec (padded
    to whole blocks, cropped back)."""
    x = synth.ar1_image(seed, H, W, 0.95, bits)
    y = O.codec_image_any_size(x, q * (1 << (bits - 8)), r, bits)["recon"]
    return x, y.astype(x.dtype)


def _run(tx, pairs, bits_list, want_map=True):
    import torch

    keep, da, db = [], [], []
    for (x, y), bits in zip(pairs, bits_list):
        tx_, vx = _dev(x, bits)
        ty_, vy = _dev(y, bits)
        keep += [tx_, ty_]
        da.append(tx.image(vx, bits))
        db.append(tx.image(vy, bits))
    n = len(pairs)
    ms = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
    total = sum((x.shape[0] - 10) * (x.shape[1] - 10) for x, _ in pairs)
    mp = torch.full((total,), -7.0, dtype=torch.float32, device="cuda") if want_map else None
    tx.tx16_ssim(da, db, ms, mp)
    torch.cuda.synchronize()
    maps = []
    if want_map:
        m = mp.cpu().numpy().astype(np.float64)
        off = 0
        for x, _ in pairs:
            h, w = x.shape[0] - 10, x.shape[1] - 10
            maps.append(m[off:off + h * w].reshape(h, w))
            off += h * w
    return ms.cpu().numpy(), maps


def _check(pair, bits, mssim, smap):
    x, y = pair
    want = O.ssim_map(x, y, bits)
    b = _bound(x, y, bits)
    assert smap.shape == want.shape
    err = np.abs(smap - want)
    assert np.all(err <= b), f"max excess {np.max(err - b)} at {np.unravel_index(np.argmax(err - b), b.shape)}"
    assert abs(mssim - want.mean()) <= b.mean() + 72 * U


SIZES = [((11, 11), 8), ((64, 64), 8), ((75, 140), 8), ((300, 47), 8), ((270, 300), 8),
         ((37, 50), 10), ((41, 33), 12)]


@pytest.mark.parametrize("shape,bits", SIZES)
def test_ssim_map_and_mean(tx, shape, bits):
    H, W = shape
    pair = _pair(500 + H + W + bits, H, W, bits)
    ms, maps = _run(tx, [pair], [bits])
    _check(pair, bits, ms[0], maps[0])


def test_ssim_identity_and_symmetry(tx):
    x, y = _pair(77, 96, 130, 8)
    ms, maps = _run(tx, [(x, x), (x, y), (y, x)], [8, 8, 8])
    assert np.all(np.abs(maps[0] - 1.0) <= 16 * U)
    assert abs(ms[0] - 1.0) <= 1e-6
    assert abs(ms[1] - ms[2]) <= 1e-6


def test_ssim_mixed_batch_without_map(tx):
    """Several images of different sizes and depths in one call; the mean
    without the map output equals the mean with it."""
    specs = [((120, 200), 8), ((33, 64), 10), ((16, 16), 8), ((300, 290), 8), ((50, 70), 12)]
    pairs = [_pair(900 + i, h, w, b) for i, ((h, w), b) in enumerate(specs)]
    bits = [b for _, b in specs]
    ms, maps = _run(tx, pairs, bits, want_map=True)
    ms2, _ = _run(tx, pairs, bits, want_map=False)
    for i in range(len(pairs)):
        _check(pairs[i], bits[i], ms[i], maps[i])
        assert abs(ms[i] - ms2[i]) <= 1e-12


def test_ssim_1080p_frame(tx):
    """One real 1920 x 1080 frame against the oracle: every position."""
    pair = _pair(4243, 1080, 1920, 8)
    ms, maps = _run(tx, [pair], [8])
    _check(pair, 8, ms[0], maps[0])


def test_ssim_rejects_bad_arguments(tx):
    import torch

    t = torch.zeros((20, 32), dtype=torch.uint8, device="cuda")
    ms = torch.zeros(1, dtype=torch.float64, device="cuda")
    small = tx.image(t[:10, :16], 8)
    with pytest.raises(tx.Tx16Error):
        tx.tx16_ssim([small], [small], ms)
    a = tx.image(t[:, :20], 8)
    b = tx.image(t[:, :21], 8)
    with pytest.raises(tx.Tx16Error):
        tx.tx16_ssim([a], [b], ms)
    tx.tx16_ssim([], [], ms)  # empty batch
