"""Shared test helpers: device upload/download of sample planes and the
oracle's per-block reference for sampled blocks."""
import numpy as np

from oracle import tx16_oracle as O


def to_dev(img: np.ndarray, pad: int = 0):
    """Upload a uint8/uint16 plane to the GPU, optionally with `pad` extra
    samples per row (a pitched view)."""
    import torch

    a = img.view(np.int16) if img.dtype == np.uint16 else img
    H, W = a.shape
    t = torch.zeros((H, W + pad), dtype=torch.from_numpy(a[:1, :1].copy()).dtype, device="cuda")
    t[:, :W] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t[:, :W]


def from_dev(t, bits: int) -> np.ndarray:
    a = t.cpu().contiguous().numpy()
    return a.view(np.uint16) if bits > 8 else a


def empty_like_img(H: int, W: int, bits: int, pad: int = 0):
    import torch

    dt = torch.uint8 if bits == 8 else torch.int16
    return torch.zeros((H, W + pad), dtype=dt, device="cuda")[:, :W]


def oracle_blocks(blocks: np.ndarray, q, r: int, bits: int) -> dict:
    """Oracle codec on a set of blocks (n, 16, 16): coefficients, levels in the
    GPU's decision precision (binary32 for q > 0, exact otherwise) and the
    reconstructed samples; plus the float64 reconstruction for tolerances."""
    X = np.asarray(blocks, dtype=np.int64)
    Y = O.forward_direct(X)
    out = {"Y": Y}
    if q is not None and q > 0:
        q = float(np.float32(q))  # the C-ABI's step is a binary32 value
    if q is None or q <= 0:
        out["levels"] = np.where(O.zonal_mask(r), Y, 0)
        out["recon"] = O.pixels_from_exact(O.inverse_exact_zonal(Y, r), bits)
        out["recon64"] = out["recon"]
        out["X64"] = O.inverse_exact_zonal(Y, r) / 256.0
    else:
        L32 = O.quantise(Y, q, r, "fp32")
        out["levels"] = L32
        out["levels64"] = O.quantise(Y, q, r, "fp64")
        out["recon"] = O.pixels_from_float(O.inverse_fp32(L32, q).astype(np.float64), bits)
        # float64 inverse of the SAME levels: isolates the binary32 inverse
        X64 = O.inverse_fp64(O.dequantise(L32, q))
        out["X64"] = X64
        out["recon64"] = O.pixels_from_float(X64, bits)
        # the float64 definition end to end (levels decided in float64 too)
        out["recon_def"] = O.pixels_from_float(
            O.inverse_fp64(O.dequantise(out["levels64"], q)), bits)
        out["c"] = np.outer(O.S_DIAG, O.S_DIAG) * Y / q
        # binary32 error bound of the inverse: at most ~34 rounded operations
        # along any path (Higham-style gamma_n times the absolute sum)
        Ta = np.abs(O.T).astype(np.float64)
        Wabs = np.abs(O.dequantise(L32, q))
        out["Xbound"] = 40 * 2.0 ** -24 * np.matmul(np.matmul(Ta.T, Wabs), Ta) + 1e-12
    return out
