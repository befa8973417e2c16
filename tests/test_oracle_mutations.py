"""Plant plausible mistakes in fresh copies of the oracle (on the CPU) and show
that the pins of ``test_oracle_pins.py`` catch every one of them."""
import importlib.util
import os

import numpy as np
import pytest

import test_oracle_pins as pins

ORACLE_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "oracle", "tx16_oracle.py")


def fresh_oracle():
    spec = importlib.util.spec_from_file_location("tx16_oracle_mutant", ORACLE_PATH)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _flip_T_sign(m):
    m.T = m.T.copy()
    m.T[6, 5] = -m.T[6, 5]


def _swap_S_entries(m):
    m.S_DIAG = m.S_DIAG.copy()
    m.S_DIAG[[2, 3]] = m.S_DIAG[[3, 2]]


def _reverse_P1(m):
    m.P1_CYCLES = [tuple(reversed(c)) for c in m.P1_CYCLES]


def _M3_plus_identity(m):
    orig = m.factor_matrices

    def fm():
        F = orig()
        F["M3"] = F["M3"].copy()
        F["M3"][4:8, 4:8] = np.eye(4, dtype=np.int64)
        return F
    m.factor_matrices = fm


def _transposed_forward(m):
    m.forward_direct = lambda blocks: np.matmul(np.matmul(m.T.T, np.asarray(blocks, np.int64)), m.T)


def _zigzag_wrong_direction(m):
    def zz(n=16):
        out = []
        for d in range(2 * n - 1):
            cells = [(u, d - u) for u in range(n) if 0 <= d - u < n]
            if d % 2 == 1:
                cells.reverse()
            out.extend(cells)
        return out
    m.zigzag_order = zz


def _bankers_rounding(m):
    m.round_half_away = lambda x: np.round(np.asarray(x, dtype=np.float64))


def _quantiser_divides_by_s(m):
    orig = m.quantise

    def q(Y, qq, r, precision="fp64"):
        saved = m.S_DIAG
        m.S_DIAG = 1.0 / saved / 16.0
        try:
            return orig(Y, qq, r, precision)
        finally:
            m.S_DIAG = saved
    m.quantise = q


def _exact_inverse_wrong_D(m):
    def inv(Y, r):
        Dp = np.rint(4.0 * m.S_DIAG).astype(np.int64)  # 4 S (rounded) instead of 16 S^2
        mask = m.zonal_mask(r)
        Wn = np.where(mask, np.asarray(Y, np.int64) * np.outer(Dp, Dp), 0)
        return np.matmul(np.matmul(m.T.T, Wn), m.T)
    m.inverse_exact_zonal = inv


def _psnr_peak_256(m):
    import math

    def p(s, H, W, bits):
        if s == 0:
            return math.inf
        return 10 * math.log10((1 << bits) ** 2 * H * W / s)
    m.psnr = p


def _dequantise_drops_q(m):
    m.dequantise = lambda levels, q: np.outer(m.S_DIAG, m.S_DIAG) * np.asarray(levels, np.float64)


def _dct_without_dc_norm(m):
    def C(n=16):
        k = np.arange(n)
        return np.sqrt(2.0 / n) * np.cos(np.pi * (2 * k[None, :] + 1) * k[:, None] / (2 * n))
    m.dct_matrix = C


def _coding_gain_arith_mean(m):
    def cg(A, rho=0.95):
        RY = A @ m.ar1_covariance(rho, A.shape[0]) @ A.T
        v = np.diag(RY)
        return float(10 * np.log10(np.mean(v) / np.mean(v * 0.9)))
    m.coding_gain = cg


def _inverse_fp32_rows_use_T(m):
    def wrong(x):
        y, _ = m.t16_factored(np.rint(np.asarray(x, np.float64)).astype(np.int64))
        return y.astype(np.float32)
    m.t16_transpose_factored_fp32 = wrong


def _blocks_column_order(m):
    def split(img):
        H, W = img.shape
        b = img.reshape(H // 16, 16, W // 16, 16).transpose(2, 0, 1, 3)
        return b.reshape(-1, 16, 16)
    m.image_to_blocks = split


def _m1_wrong_half(m):
    orig = m._butterfly

    def bf(n):
        B = orig(n)
        if n == 16:
            B = B.copy()
            B[8:, 8:] = -B[8:, 8:]  # +I8 where the paper has -I8
        return B
    m._butterfly = bf


def _ssim_k2_too_large(m):
    m.SSIM_K2 = 0.3


def _ssim_structure_drops_two(m):
    orig = m.window_mean

    def ssim_map(x, y, bits=8):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        L = float((1 << bits) - 1)
        C1, C2 = (m.SSIM_K1 * L) ** 2, (m.SSIM_K2 * L) ** 2
        w = m.ssim_window()
        mx, my = orig(x, w), orig(y, w)
        sxx = orig(x * x, w) - mx * mx
        syy = orig(y * y, w) - my * my
        sxy = orig(x * y, w) - mx * my
        return ((2 * mx * my + C1) * (sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    m.ssim_map = ssim_map


def _ssim_sigma_one(m):
    m.SSIM_SIGMA = 1.0
    orig = m.ssim_window
    m.ssim_window = lambda size=11, sigma=1.0: orig(size, sigma)


def _ssim_raw_second_moments(m):
    orig = m.window_mean

    def ssim_map(x, y, bits=8):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        L = float((1 << bits) - 1)
        C1, C2 = (m.SSIM_K1 * L) ** 2, (m.SSIM_K2 * L) ** 2
        w = m.ssim_window()
        mx, my = orig(x, w), orig(y, w)
        sxx, syy, sxy = orig(x * x, w), orig(y * y, w), orig(x * y, w)  # means not subtracted
        return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    m.ssim_map = ssim_map


def _ssim_window_unnormalised(m):
    orig = m.ssim_window
    m.ssim_window = lambda size=11, sigma=1.5: orig(size, sigma) * 2 * np.pi * sigma * sigma


def _ssim_window_one_column_late(m):
    def wm(img, w):
        img = np.asarray(img, dtype=np.float64)
        k = w.shape[0]
        H, W = img.shape
        out = np.zeros((H - k + 1, W - k))
        for a in range(k):
            for b in range(k):
                out += w[a, b] * img[a:a + H - k + 1, b + 1:b + 1 + W - k]
        return out
    m.window_mean = wm


def _ssim_peak_256(m):
    def ssim_map(x, y, bits=8):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        L = float(1 << bits)  # 2^bits where the peak is 2^bits - 1
        C1, C2 = (m.SSIM_K1 * L) ** 2, (m.SSIM_K2 * L) ** 2
        w = m.ssim_window()
        mx, my = m.window_mean(x, w), m.window_mean(y, w)
        sxx = m.window_mean(x * x, w) - mx * mx
        syy = m.window_mean(y * y, w) - my * my
        sxy = m.window_mean(x * y, w) - mx * my
        return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    m.ssim_map = ssim_map


def _t8_wrong_output_order(m):
    orig = m.t8_output_order
    m.t8_output_order = lambda: (lambda g: [g[0], g[2], g[1]] + g[3:])(orig())


def _s8_squared(m):
    orig = m.s8_diag
    m.s8_diag = lambda: orig() ** 2 * 2.0


def _codec8_transposed(m):
    m.forward8 = lambda blocks: np.matmul(np.matmul(m.t8_matrix().T, np.asarray(blocks, np.int64)), m.t8_matrix())


def _mixed_ties_to_8(m):
    orig = m.codec_image_mixed

    def mixed(img, q, r16, r8, bits=8, mode="auto", precision="fp64"):
        res = orig(img, q, r16, r8, bits, mode, precision)
        if mode != "auto":
            return res
        a16 = orig(img, q, r16, r8, bits, "16", precision)["recon"]
        a8 = orig(img, q, r16, r8, bits, "8", precision)["recon"]
        x = np.asarray(img, np.int64)
        H, W = x.shape
        e16 = ((x - a16) ** 2).reshape(H // 16, 16, W // 16, 16).sum(axis=(1, 3))
        e8 = ((x - a8) ** 2).reshape(H // 16, 16, W // 16, 16).sum(axis=(1, 3))
        split = e8 <= e16
        sel = np.kron(split, np.ones((16, 16), dtype=bool))
        rec = np.where(sel, a8, a16)
        return {"recon": rec, "split": split, "sse": m.sse(x, rec), "psnr": 0.0}
    m.codec_image_mixed = mixed


MUTANTS = [_flip_T_sign, _swap_S_entries, _reverse_P1, _M3_plus_identity,
           _transposed_forward, _zigzag_wrong_direction, _bankers_rounding,
           _quantiser_divides_by_s, _exact_inverse_wrong_D, _psnr_peak_256,
           _dequantise_drops_q, _dct_without_dc_norm, _coding_gain_arith_mean,
           _inverse_fp32_rows_use_T, _blocks_column_order, _m1_wrong_half,
           _ssim_k2_too_large, _ssim_structure_drops_two, _ssim_sigma_one, _ssim_raw_second_moments,
           _ssim_window_unnormalised, _ssim_window_one_column_late, _ssim_peak_256,
           _t8_wrong_output_order, _s8_squared, _codec8_transposed, _mixed_ties_to_8]


@pytest.mark.parametrize("mutate", MUTANTS, ids=[f.__name__.strip("_") for f in MUTANTS])
def test_planted_mistake_is_caught(mutate):
    m = fresh_oracle()
    mutate(m)
    failed = []
    for check in pins.ALL_CHECKS:
        try:
            check(m)
        except Exception:  # noqa: BLE001 - any failure counts as caught
            failed.append(check.__name__)
    assert failed, f"no pin caught mutation {mutate.__name__}"


def test_unmutated_copy_passes_every_pin():
    m = fresh_oracle()
    for check in pins.ALL_CHECKS:
        check(m)
