"""Pins of the CPU oracle to facts the paper and mathematics fix.

Each ``check_*`` function takes the oracle module, so that
``test_oracle_mutations.py`` can run the same checks against deliberately
broken copies of it and show that every plausible mistake fails one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

from oracle import tx16_oracle as O
from paper_1606_07414_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                out[line[0]] = [float(v) for v in line[1:]]
    return out


def _golden_ints(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            vals += [int(v) for v in line.split("#")[0].split()]
    return vals


# ----------------------------------------------------------------------------
# Sec. 2.1: T, S, C_hat
# ----------------------------------------------------------------------------
def check_T_gram_matches_printed_S(o):
    """Two printed items agree: S (printed) == sqrt((T T^t)^-1) from the
    printed T, via scipy's matrix square root; T T^t is diagonal."""
    Tm = o.T.astype(np.float64)
    assert set(np.unique(o.T)) <= {-1, 0, 1}
    G = Tm @ Tm.T
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0, "T T^t not diagonal"
    S_from_T = scipy.linalg.sqrtm(np.linalg.inv(G)).real
    np.testing.assert_allclose(S_from_T, np.diag(o.S_DIAG), atol=1e-14)


def check_c_hat_orthogonal(o):
    C = o.c_hat()
    np.testing.assert_allclose(C @ C.T, np.eye(16), atol=1e-14)


def check_factor_product_is_T(o):
    F = o.factor_matrices()
    P = np.eye(16, dtype=np.int64)
    for name in o.FACTOR_ORDER:
        P = F[name] @ P
    assert np.array_equal(P, o.T), "P2 M4 M3 M2 P1 M1 != T"


def check_addition_counts(o):
    """Table 1: 44 additions (16 + 16 + 8 + 4), 0 multiplications; direct 112."""
    g = _golden_kv("table1_complexity.txt")
    F = o.factor_matrices()
    per_stage = [o.stage_additions(F[n]) for n in o.FACTOR_ORDER]
    assert per_stage == [16, 0, 16, 8, 4, 0]
    assert sum(per_stage) == g["proposed_add"][0]
    assert o.stage_additions(o.T) == g["direct_add"][0]
    # counted while running, too
    _, adds = o.t16_factored(np.arange(16))
    assert adds == g["proposed_add"][0]
    for key, other in (("saving_vs_60", 60), ("saving_vs_64", 64), ("saving_vs_72", 72)):
        assert round(100 * (1 - adds / other), 2) == g[key][0]


def check_factored_equals_direct_1d(o):
    """Linearity makes the 16 unit vectors an exhaustive proof; add brute force
    over {0,1}^16 and 10,000 seeded random vectors (the hardware test size of
    Sec. 4)."""
    E = np.eye(16, dtype=np.int64)
    y, _ = o.t16_factored(E)  # row j of E -> T e_j
    assert np.array_equal(y.T, o.T)
    bits = ((np.arange(1 << 16)[:, None] >> np.arange(16)[None, :]) & 1).astype(np.int64)
    y, _ = o.t16_factored(bits)
    assert np.array_equal(y, bits @ o.T.T)
    x = (synth.splitmix64(2016, 16 * 10000) % np.uint64(2048)).astype(np.int64).reshape(-1, 16) - 1024
    y, _ = o.t16_factored(x)
    assert np.array_equal(y, x @ o.T.T)


def check_forward_2d(o):
    """Factored == direct on random 8- and 10-bit blocks; DC is the block sum
    (row 0 of T is all ones); a block that varies only along its rows
    (horizontally) has energy only in row u = 0 of Y, and one that varies only
    down its columns only in column v = 0 (B = C A C^t transforms columns of A
    on the left and rows on the right)."""
    for bits in (8, 10):
        X = (synth.splitmix64(7 + bits, 64 * 256) % np.uint64(1 << bits)).astype(np.int64)
        X = X.reshape(64, 16, 16)
        Yd = o.forward_direct(X)
        assert np.array_equal(Yd, o.forward_factored(X))
        assert np.array_equal(Yd[:, 0, 0], X.sum(axis=(1, 2)))
    row = np.arange(16, dtype=np.int64) * 13 % 251
    horiz = np.broadcast_to(row[None, :], (16, 16))
    Y = o.forward_direct(horiz[None])[0]
    assert np.any(Y[0, 1:] != 0) and np.all(Y[1:, :] == 0)
    Y = o.forward_direct(horiz.T[None])[0]
    assert np.any(Y[1:, 0] != 0) and np.all(Y[:, 1:] == 0)
    # magnitude bound used for int32 kernels: 256 * max|x|
    ext = np.full((1, 16, 16), 255, dtype=np.int64)
    assert np.abs(o.forward_direct(ext)).max() == 255 * 256


# ----------------------------------------------------------------------------
# Sec. 2.3, Table 2
# ----------------------------------------------------------------------------
def check_exact_dct_is_textbook(o):
    """The exact DCT-II of Table 2 is scipy's orthonormal DCT-II."""
    ref = scipy.fft.dct(np.eye(16), type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(o.dct_matrix(16), ref, atol=1e-14)


def check_table2(o):
    g = _golden_kv("table2_proposed.txt")
    C = o.c_hat()
    got = [o.dct_distortion(C), o.total_error_energy(C), o.transform_mse(C),
           o.coding_gain(C), o.transform_efficiency(C)]
    for name, want, have in zip(("d2", "eps", "mse", "cg", "eta"), g["proposed"], got):
        assert round(have, 3) == pytest.approx(want, abs=1e-9), (name, have, want)
    D = o.dct_matrix(16)
    got = [o.dct_distortion(D), o.total_error_energy(D), o.transform_mse(D),
           o.coding_gain(D), o.transform_efficiency(D)]
    for name, want, have in zip(("d2", "eps", "mse", "cg", "eta"), g["exact_dct"], got):
        assert abs(round(have, 3)) == pytest.approx(want, abs=1e-9), (name, have, want)


# ----------------------------------------------------------------------------
# Sec. 3.1 codec
# ----------------------------------------------------------------------------
def check_zigzag_matches_jpeg(o):
    want = _golden_ints("jpeg_zigzag8.txt")
    assert [u * 8 + v for (u, v) in o.zigzag_order(8)] == want
    zz = o.zigzag_order(16)
    assert len(set(zz)) == 256
    # the 16x16 scan restricted to the first 36 cells (the triangle shared
    # with the 8x8 scan) is the JPEG scan
    assert [(u, v) for (u, v) in zz[:36]] == [(k // 8, k % 8) for k in want[:36]]


def check_zonal_is_prefix_per_column(o):
    """Inside each column v the kept rows are a prefix 0..m_v-1, and the zone
    grows by exactly one cell per step of r."""
    prev = 0
    for r in range(1, 257):
        m = o.zonal_mask(r)
        assert m.sum() == r
        for v in range(16):
            col = m[:, v]
            k = col.sum()
            assert col[:k].all() and not col[k:].any()
        assert m.sum() - prev == 1
        prev = m.sum()


def check_blocks_roundtrip(o):
    img = np.arange(48 * 32, dtype=np.int64).reshape(48, 32)
    b = o.image_to_blocks(img)
    assert b.shape == (6, 16, 16)
    assert np.array_equal(b[3], img[16:32, 16:32])  # raster block order
    assert np.array_equal(o.blocks_to_image(b, 48, 32), img)


def check_perfect_reconstruction(o):
    """r = 256 with no quantiser reconstructs exactly: C_hat^t C_hat X C_hat^t
    C_hat = X by orthogonality (Sec. 2.1), here as the integer identity
    256 X = T^t (D' Y D') T."""
    for bits in (8, 10):
        img = synth.ar1_image(3 + bits, 64, 48, 0.95, bits).astype(np.int64)
        X = o.image_to_blocks(img)
        Y = o.forward_direct(X)
        num = o.inverse_exact_zonal(Y, 256)
        assert np.array_equal(num, 256 * X)
        res = o.codec_image(img, None, 256, bits)
        assert res["sse"] == 0 and res["psnr"] == math.inf
        res = o.codec_image(img, None, 256, bits, forward="factored")
        assert res["sse"] == 0 and np.array_equal(res["Y"], Y)


def check_dc_only_is_block_mean(o):
    """r = 1 keeps only DC: every pixel of a block becomes the rounded block
    mean (closed form), with no quantiser and with a tiny power-of-two q."""
    img = synth.ar1_image(11, 64, 64, 0.9).astype(np.int64)
    X = o.image_to_blocks(img)
    mean = X.sum(axis=(1, 2)) / 256.0
    want = np.sign(mean) * np.floor(np.abs(mean) + 0.5)
    for q, prec in ((None, "fp64"), (2.0 ** -12, "fp64"), (2.0 ** -12, "fp32")):
        rec = o.image_to_blocks(o.codec_image(img, q, 1, 8, prec)["recon"])
        assert np.array_equal(rec, np.broadcast_to(want[:, None, None], rec.shape)), (q, prec)


def check_quantiser_limits(o):
    img = synth.ar1_image(12, 32, 64, 0.95).astype(np.int64)
    for prec in ("fp64", "fp32"):
        res = o.codec_image(img, 2.0 ** -8, 256, 8, prec)
        assert res["sse"] == 0, prec  # step -> 0 recovers X
        res = o.codec_image(img, 1e9, 256, 8, prec)
        assert np.all(res["levels"] == 0) and res["sse"] == int(np.sum(img * img)), prec


def check_quantiser_scaling(o):
    """level = round(s_u s_v Y / q): checked on constructed coefficients whose
    orthonormal value is an exact half-integer multiple of q (ties away from
    zero) and against the class of each (u, v) (d_u d_v / 16)."""
    d = np.array([1, 1, 2, 2 ** 0.5, 2 ** 0.5, 1, 2, 2, 1, 2, 2, 2 ** 0.5, 2 ** 0.5, 2, 2, 2])
    Y = np.zeros((1, 16, 16), dtype=np.int64)
    Y[0, 0, 0] = 40   # c = 40/16 = 2.5 -> q=1 -> 3
    Y[0, 0, 2] = -20  # c = -20*2/16 = -2.5 -> -3
    Y[0, 2, 6] = 9    # c = 9*4/16 = 2.25 -> 2
    Y[0, 3, 4] = 8    # c = 8*2/16 = 1 -> 1
    Y[0, 3, 0] = 16   # c = 16*sqrt2/16 = 1.414 -> 1
    for prec in ("fp64", "fp32"):
        L = o.quantise(Y, 1.0, 256, prec)[0]
        assert (L[0, 0], L[0, 2], L[2, 6], L[3, 4], L[3, 0]) == (3, -3, 2, 1, 1), prec
    c = np.outer(d, d) / 16.0
    np.testing.assert_allclose(np.outer(o.S_DIAG, o.S_DIAG), c, rtol=1e-15)


def check_fp32_decisions_only_differ_at_near_ties(o):
    img = synth.ar1_image(21, 128, 128, 0.95).astype(np.int64)
    X = o.image_to_blocks(img)
    Y = o.forward_direct(X)
    for q, r in ((16.0, 64), (8.0, 16), (32.0, 256), (5.3, 100)):
        L64 = o.quantise(Y, q, r, "fp64")
        L32 = o.quantise(Y, q, r, "fp32")
        c = np.outer(o.S_DIAG, o.S_DIAG) * Y / q
        diff = L64 != L32
        assert np.all(np.abs(L64 - L32) <= 1)
        assert np.all(np.abs(np.abs(c[diff]) - np.floor(np.abs(c[diff])) - 0.5) < 1e-5)
        X64 = o.inverse_fp64(o.dequantise(L32, q))
        X32 = o.inverse_fp32(L32, q).astype(np.float64)
        # Higham-style bound for at most ~34 rounded operations along any path
        Wabs = np.abs(o.dequantise(L32, q))
        Ta = np.abs(o.T).astype(np.float64)
        bound = 40 * 2.0 ** -24 * np.matmul(np.matmul(Ta.T, Wabs), Ta) + 1e-12
        assert np.all(np.abs(X64 - X32) <= bound)
        p64 = o.pixels_from_float(X64, 8)
        p32 = o.pixels_from_float(X32, 8)
        bad = p64 != p32
        assert np.all(np.abs(p64 - p32) <= 1)
        assert np.all(np.abs(np.abs(X64[bad]) % 1.0 - 0.5) <= bound[bad])


def check_rounding(o):
    x = np.array([0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 0.49999997, -0.49999997, 3.7, -3.7])
    assert list(o.round_half_away(x)) == [1, -1, 2, -2, 3, -3, 0, 0, 4, -4]
    x32 = np.float32(0.49999997)
    assert o.round_half_away(np.array([x32]))[0] == 0.0


def check_psnr_closed_forms(o):
    assert o.psnr(0, 16, 16, 8) == math.inf
    # an error of exactly 1 at every pixel: PSNR = 20 log10(peak)
    assert o.psnr(512 * 512, 512, 512, 8) == pytest.approx(20 * math.log10(255), abs=1e-12)
    assert o.psnr(64 * 32, 32, 64, 10) == pytest.approx(20 * math.log10(1023), abs=1e-12)
    # error 4 everywhere: 12.04 dB lower
    assert o.psnr(16 * 256, 16, 16, 8) == pytest.approx(20 * math.log10(255 / 4), abs=1e-12)
    a = np.array([[0, 10], [255, 7]])
    b = np.array([[3, 10], [250, 9]])
    assert o.sse(a, b) == 9 + 25 + 4


def check_any_size_codec(o):
    """Edge replication: on sizes that are multiples of 16 it is the plain
    codec; otherwise the padded pixels repeat the last row/column (numpy's
    edge mode, a library routine) and the error counts original pixels only."""
    img = synth.ar1_image(31, 48, 64, 0.95).astype(np.int64)
    a = o.codec_image_any_size(img, 16.0, 16, 8, "fp32")
    b = o.codec_image(img, 16.0, 16, 8, "fp32")
    assert np.array_equal(a["recon"], b["recon"]) and a["sse"] == b["sse"]
    odd = synth.ar1_image(32, 37, 50, 0.95).astype(np.int64)
    P = o.pad_to_blocks(odd)
    assert P.shape == (48, 64)
    assert np.array_equal(P[:37, :50], odd)
    assert np.all(P[37:, :50] == odd[36]) and np.all(P[:37, 50:] == odd[:, 49:50])
    assert np.all(P[37:, 50:] == odd[36, 49])
    c = o.codec_image_any_size(odd, None, 256, 8)  # lossless zone: exact on any size
    assert c["sse"] == 0 and c["recon"].shape == odd.shape
    d = o.codec_image_any_size(odd, 16.0, 4, 8, "fp32")
    full = o.codec_image(P, 16.0, 4, 8, "fp32")
    assert np.array_equal(d["recon"], full["recon"][:37, :50])
    assert d["psnr"] == o.psnr(o.sse(odd, d["recon"]), 37, 50, 8)


# ----------------------------------------------------------------------------
# Sec. 2.1 and Sec. 3.2: T8, the 8-point approximation T is built from
# ----------------------------------------------------------------------------
def check_t8_from_factorisation(o):
    """T8 from the first half of M2 M3 M4 equals the printed T's even rows on
    the first 8 columns; it costs 8 + 4 + 2 = 14 additions, the count Sec. 2.1
    quotes for the 8-point approximation; the network equals the matrix on
    every {0,1}^8 input; T on a symmetric input gives 2 T8 x on its even rows
    and zero on its odd rows."""
    T8 = o.t8_matrix()
    assert T8.shape == (8, 8)
    assert np.array_equal(T8, o.T[0::2, :8])
    assert [o.stage_additions(M) for _, M in o.t8_stages()] == [8, 4, 2]
    X = np.array([[(k >> j) & 1 for j in range(8)] for k in range(256)], dtype=np.int64)
    y, adds = o.t8_factored(X)
    assert adds == 14
    assert np.array_equal(y, X @ T8.T)
    rng = np.random.default_rng(8)
    x8 = rng.integers(-255, 256, (50, 8))
    y16 = np.concatenate([x8, x8[:, ::-1]], axis=1) @ o.T.T
    assert np.array_equal(y16[:, 0::2], 2 * (x8 @ T8.T))
    assert not np.any(y16[:, 1::2])
    # transposed network in binary32 on small integers (exact) and on reals
    z = rng.integers(-1000, 1000, (64, 8)).astype(np.float32)
    assert np.array_equal(o.t8_transpose_factored_fp32(z).astype(np.float64), z.astype(np.float64) @ T8)
    zr = rng.normal(0, 100, (64, 8)).astype(np.float32)
    assert np.allclose(o.t8_transpose_factored_fp32(zr), zr.astype(np.float64) @ T8, rtol=1e-5, atol=1e-3)


def check_s8(o):
    """T8 T8^t is diagonal; S8 relates to the printed S by S[2k] = S8[k]/sqrt2
    (the even rows of T see each sum twice); C8 = S8 T8 is orthogonal."""
    s8 = o.s8_diag()
    assert np.allclose(o.S_DIAG[0::2], s8 / math.sqrt(2), rtol=1e-15)
    C8 = np.diag(s8) @ o.t8_matrix()
    assert np.allclose(C8 @ C8.T, np.eye(8), atol=1e-14)


def check_codec8(o):
    """8 x 8 codec: lossless with all 64 cells and no quantiser; r = 1 gives
    the block mean; the binary32 and float64 paths agree away from ties."""
    blocks = o.image_to_blocks8(synth.ar1_image(81, 32, 48, 0.9).astype(np.int64))
    assert np.array_equal(o.codec_blocks8(blocks, None, 64), blocks)
    mean = o.round_half_away(blocks.mean(axis=(1, 2)))
    r1 = o.codec_blocks8(blocks, None, 1)
    assert np.array_equal(r1, np.broadcast_to(mean[:, None, None], r1.shape))
    img = synth.ar1_image(82, 48, 64, 0.95).astype(np.int64)
    b = o.image_to_blocks8(img)
    assert np.array_equal(o.blocks8_to_image(b, 48, 64), img)
    # levels: binary32 and float64 decisions differ by one at most, and only
    # where c / q lies within a few binary32 ulps of a rounding tie
    Y = o.forward8(b)
    L32, L64 = o.quantise8(Y, 16.0, 10, "fp32"), o.quantise8(Y, 16.0, 10, "fp64")
    t = np.abs(np.outer(o.s8_diag(), o.s8_diag()) * Y / 16.0)
    d = L32 != L64
    assert np.all(np.abs(L32 - L64) <= 1)
    assert np.all(np.abs(t[d] - np.floor(t[d]) - 0.5) <= 2.0 ** -22 * t[d])
    # the same levels reconstruct to the same samples in both precisions
    # unless the float64 value lies near a rounding tie
    X32 = o.inverse8_fp32(L64, 16.0).astype(np.float64)
    X64 = o.inverse8_fp64(L64, 16.0)
    p32, p64 = o.pixels_from_float(X32, 8), o.pixels_from_float(X64, 8)
    far = np.abs(np.abs(X64) % 1.0 - 0.5) > 1e-3
    assert np.array_equal(p32[far], p64[far])
    assert np.max(np.abs(X32 - X64)) < 1e-3


def check_mixed_codec(o):
    """Mixed tiling: forcing 16 x 16 is the plain codec, forcing 8 x 8 is the
    8 x 8 codec, and the automatic choice keeps, per region, the tiling with
    the smaller squared error (so its total is at most either forced one)."""
    img = synth.ar1_image(83, 48, 64, 0.95).astype(np.int64)
    m16 = o.codec_image_mixed(img, 16.0, 16, 4, 8, "16", "fp32")
    assert np.array_equal(m16["recon"], o.codec_image(img, 16.0, 16, 8, "fp32")["recon"])
    m8 = o.codec_image_mixed(img, 16.0, 16, 4, 8, "8", "fp32")
    want8 = o.blocks8_to_image(o.codec_blocks8(o.image_to_blocks8(img), 16.0, 4, 8, "fp32"), 48, 64)
    assert np.array_equal(m8["recon"], want8)
    ma = o.codec_image_mixed(img, 16.0, 16, 4, 8, "auto", "fp32")
    assert ma["sse"] <= min(m16["sse"], m8["sse"])
    # flat regions reconstruct exactly either way: a tie, kept as 16 x 16
    flat = np.full((32, 32), 77, dtype=np.int64)
    mf = o.codec_image_mixed(flat, None, 1, 1, 8, "auto")
    assert mf["sse"] == 0 and not np.any(mf["split"])
    for by in range(3):
        for bx in range(4):
            sl = (slice(16 * by, 16 * by + 16), slice(16 * bx, 16 * bx + 16))
            e16 = o.sse(img[sl], m16["recon"][sl])
            e8 = o.sse(img[sl], m8["recon"][sl])
            assert bool(ma["split"][by, bx]) == (e8 < e16)
            assert np.array_equal(ma["recon"][sl], m8["recon"][sl] if e8 < e16 else m16["recon"][sl])


# ----------------------------------------------------------------------------
# SSIM (Sec. 3.1, Fig. 2(b); Wang et al. 2004 window and constants)
# ----------------------------------------------------------------------------
def check_ssim_window(o):
    """The window is scipy's 11-point Gaussian of standard deviation 1.5, as
    an outer product, normalised to unit sum; the local means are scipy's
    'valid' 2-D correlation with it."""
    import scipy.signal

    w = o.ssim_window()
    g = scipy.signal.windows.gaussian(11, std=1.5)
    ref = np.outer(g, g) / np.outer(g, g).sum()
    assert w.shape == (11, 11)
    assert np.allclose(w, ref, rtol=1e-14, atol=0)
    img = synth.ar1_image(41, 30, 27, 0.9).astype(np.float64)
    got = o.window_mean(img, w)
    want = scipy.signal.correlate2d(img, ref, mode="valid")
    assert got.shape == (20, 17)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-9)


def check_ssim_identity_symmetry_constants(o):
    x = synth.ar1_image(42, 40, 36, 0.95)
    y = o.codec_image(synth.ar1_image(42, 48, 48, 0.95)[:48, :48], 16.0, 8, 8)["recon"][:40, :36]
    assert o.ssim(x, x) == pytest.approx(1.0, abs=1e-12)
    assert o.ssim(x, y) == pytest.approx(o.ssim(y, x), abs=1e-12)
    assert o.ssim_map(x, y).shape == (30, 26)
    # constant images: the structure term is C2 / C2, the luminance term is
    # (2ab + C1) / (a^2 + b^2 + C1), C1 = (0.01 L)^2
    for a, b, bits in ((100, 140, 8), (0, 255, 8), (700, 650, 10)):
        L = (1 << bits) - 1
        C1 = (0.01 * L) ** 2
        want = (2 * a * b + C1) / (a * a + b * b + C1)
        got = o.ssim(np.full((16, 20), a), np.full((16, 20), b), bits)
        assert got == pytest.approx(want, rel=1e-12)


def check_ssim_checkerboard_closed_form(o):
    """x = m + d (-1)^(i+j), y = n + e (-1)^(i+j).  For a window at (i0, j0)
    with sign t = (-1)^(i0+j0) and s = sum_k g_k (-1)^k over the normalised
    1-D Gaussian g: mu_x = m + t d s^2, s_x^2 = d^2 (1 - s^4),
    s_xy = d e (1 - s^4); half the positions have t = +1."""
    k = np.arange(11) - 5.0
    g = np.exp(-k * k / (2 * 1.5 ** 2))
    g /= g.sum()
    s2 = float(np.sum(g * (-1.0) ** np.arange(11))) ** 2
    m, d, n, e = 120.0, 30.0, 100.0, -12.0
    H, W = 30, 40  # 20 x 30 window positions: half with each sign
    i, j = np.indices((H, W))
    sgn = (-1.0) ** (i + j)
    x = m + d * sgn
    y = n + e * sgn
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    cs = (2 * d * e * (1 - s2 * s2) + C2) / ((d * d + e * e) * (1 - s2 * s2) + C2)
    lum = [(2 * (m + t * d * s2) * (n + t * e * s2) + C1) / ((m + t * d * s2) ** 2 + (n + t * e * s2) ** 2 + C1)
           for t in (1.0, -1.0)]
    assert o.ssim(x, y) == pytest.approx(0.5 * (lum[0] + lum[1]) * cs, rel=1e-12)


def check_ssim_one_window_by_weighted_covariance(o):
    """One window position against numpy's weighted mean and weighted
    covariance (np.average, np.cov with aweights, bias=True)."""
    x = synth.ar1_image(43, 11, 11, 0.8).astype(np.float64)
    y = synth.ar1_image(44, 11, 11, 0.8).astype(np.float64)
    w = o.ssim_window().ravel()
    mx, my = np.average(x.ravel(), weights=w), np.average(y.ravel(), weights=w)
    c = np.cov(np.stack([x.ravel(), y.ravel()]), aweights=w, bias=True)
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    want = ((2 * mx * my + C1) * (2 * c[0, 1] + C2)) / ((mx * mx + my * my + C1) * (c[0, 0] + c[1, 1] + C2))
    got = o.ssim_map(x, y)
    assert got.shape == (1, 1)
    assert got[0, 0] == pytest.approx(want, rel=1e-10)


ALL_CHECKS = [v for k, v in sorted(globals().items()) if k.startswith("check_")]


@pytest.mark.parametrize("check", ALL_CHECKS, ids=[c.__name__ for c in ALL_CHECKS])
def test_oracle_pin(check):
    check(O)


def test_permutation_convention_is_the_only_one():
    """Of the four ways to read the cyclic notation (positions or values,
    sigma or its inverse) only the oracle's reproduces T."""
    F = O.factor_matrices()
    ok = 0
    for transpose_p1 in (False, True):
        for transpose_p2 in (False, True):
            P1 = F["P1"].T if transpose_p1 else F["P1"]
            P2 = F["P2"].T if transpose_p2 else F["P2"]
            prod = P2 @ F["M4"] @ F["M3"] @ F["M2"] @ P1 @ F["M1"]
            ok += int(np.array_equal(prod, O.T))
            if np.array_equal(prod, O.T):
                assert not transpose_p1 and not transpose_p2
    assert ok == 1


def test_quantiser_constants_are_far_from_binary32_midpoints():
    """f = fl32(s_u s_v / q) and g = fl32(q s_u s_v) are computed independently
    on the GPU host side; they agree only if no double value lies within a few
    double ulps of a binary32 rounding midpoint.  Check the step sizes used."""
    ss = np.unique(np.outer(O.S_DIAG, O.S_DIAG))
    for q in (1.0, 2.0, 5.3, 8.0, 10.0, 16.0, 32.0, 2.0 ** -8, 2.0 ** -12, 1e9):
        for x in np.concatenate([ss / q, ss * q]):
            f = np.float32(x)
            ulp32 = np.spacing(f)
            frac = abs(float(x) - float(f)) / float(ulp32)
            assert abs(frac - 0.5) > 1e-6, (q, x)


def test_t8_quantiser_constants_agree_with_the_library_formula():
    """The library forms the 8 x 8 constants from s8_u s8_v = 2^(-3 + k/2)
    (k = c(u) + c(v)) in double; the oracle from products of S8 entries.  The
    binary32 values agree for every step size the tests use (no double value
    within a few ulps of a binary32 midpoint)."""
    s8 = O.s8_diag()
    for q in (1.0, 2.0, 4.0, 5.3, 8.0, 12.0, 16.0, 32.0, 64.0):
        for u in range(8):
            for v in range(8):
                c = [0, 2, 1, 2, 0, 2, 1, 2]
                k = c[u] + c[v]
                lib = math.ldexp(1.0, -3 + k // 2) * (math.sqrt(2.0) if k & 1 else 1.0)
                x = s8[u] * s8[v]
                assert np.float32(x / q) == np.float32(lib / q), (q, u, v)
                assert np.float32(q * x) == np.float32(q * lib), (q, u, v)
                f = np.float32(x / q)
                assert abs(abs(float(x / q) - float(f)) / float(np.spacing(f)) - 0.5) > 1e-6
