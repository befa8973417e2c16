"""CPU oracle for the 16-point multiplierless DCT approximation codec.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain, obviously correct
restatement of what the paper computes, used to prove the CUDA path right.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code, table or constant with the
CUDA library in ``paper_1606_07414_gb300/`` and imports nothing from it;
the product path never imports this module.

Everything follows the paper (Cintra, Bayer, Oliveira et al., "Multiplierless
16-point DCT approximation for low-complexity image and video coding"):

* Sec. 2.1 -- the integer matrix T (entries in {0, +1, -1}), the diagonal
  orthogonalising matrix S = sqrt((T T^t)^-1) and C_hat = S T.
* Sec. 2.2 -- the sparse factorisation T = P2 M4 M3 M2 P1 M1 (44 additions)
  and Table 1 (cost).
* Sec. 2.3 -- Table 2 (d2, epsilon, MSE, coding gain, efficiency, AR(1)
  rho = 0.95).
* Sec. 3.1 -- the JPEG-like block codec: 16x16 blocks, B = C A C^t, keep the
  first r coefficients in zig-zag order, inverse C^t B C, PSNR.
* Sec. 2.1 (last paragraph) -- S is merged into the quantiser.

Integer work is int64, floating point is float64, except the functions named
``*_fp32``, which take the one decision the paper leaves to the implementation
-- rounding a scaled coefficient or a reconstructed pixel to an integer -- in
binary32 arithmetic, the precision of the GPU kernels (see ``quantise`` and
``inverse_fp32``).

Readings of the paper that this oracle takes where the text is silent or
garbled are stated at each function.  PSNR on the paper's own images has no
reproducible value here (the USC-SIPI images and Lena are not available):
"parity unpinned" for the paper's 25.84 dB figure; the PSNR function itself is
pinned by closed forms.
"""
from __future__ import annotations

import math

import numpy as np

N = 16

# ---------------------------------------------------------------------------
# Sec. 2.1: the transformation matrix T, as printed (rows = output index).
# ---------------------------------------------------------------------------
T = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
        [1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1, -1, -1],
        [1, 0, 0, 0, 0, 0, 0, -1, -1, 0, 0, 0, 0, 0, 0, 1],
        [1, 1, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, -1, -1],
        [1, 0, 0, -1, -1, 0, 0, 1, 1, 0, 0, -1, -1, 0, 0, 1],
        [1, 1, -1, -1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1],
        [0, 0, -1, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, -1, 0, 0],
        [0, 0, 0, 0, 0, 0, -1, 1, -1, 1, 0, 0, 0, 0, 0, 0],
        [1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1],
        [0, 0, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0, -1, 1, 0, 0],
        [0, -1, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, -1, 0],
        [0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0],
        [0, -1, 1, 0, 0, 1, -1, 0, 0, -1, 1, 0, 0, 1, -1, 0],
        [1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1],
        [0, 0, 0, -1, 1, 0, 0, 0, 0, 0, 0, 1, -1, 0, 0, 0],
        [0, 0, 0, 0, -1, 1, 0, 0, 0, 0, -1, 1, 0, 0, 0, 0],
    ],
    dtype=np.int64,
)

# Sec. 2.1: S = (1/4) diag(1, 1, 2, sqrt2, sqrt2, 1, 2, 2, 1, 2, 2, sqrt2,
# sqrt2, 2, 2, 2), as printed.  S_DIAG holds the diagonal.
_R2 = math.sqrt(2.0)
S_DIAG = 0.25 * np.array(
    [1, 1, 2, _R2, _R2, 1, 2, 2, 1, 2, 2, _R2, _R2, 2, 2, 2], dtype=np.float64
)


def c_hat() -> np.ndarray:
    """Sec. 2.1: the orthogonal approximation C_hat = S . T (float64)."""
    return np.diag(S_DIAG) @ T.astype(np.float64)


# ---------------------------------------------------------------------------
# Sec. 2.2: the sparse factorisation T = P2 . M4 . M3 . M2 . P1 . M1.
# ---------------------------------------------------------------------------
def _eye(n: int) -> np.ndarray:
    return np.eye(n, dtype=np.int64)


def _counter_eye(n: int) -> np.ndarray:
    """The counter-identity (anti-diagonal ones) of order n, written I-bar."""
    return np.fliplr(np.eye(n, dtype=np.int64))


def _butterfly(n: int) -> np.ndarray:
    """[[I_{n/2}, Ibar_{n/2}], [Ibar_{n/2}, -I_{n/2}]] -- the block that
    M1 (n = 16), M2 (n = 8) and M3 (n = 4) are built from."""
    h = n // 2
    return np.block([[_eye(h), _counter_eye(h)], [_counter_eye(h), -_eye(h)]])


def _block_diag(*blocks: np.ndarray) -> np.ndarray:
    n = sum(b.shape[0] for b in blocks)
    out = np.zeros((n, n), dtype=np.int64)
    k = 0
    for b in blocks:
        m = b.shape[0]
        out[k : k + m, k : k + m] = b
        k += m
    return out


def _cycles_to_matrix(cycles: list[tuple[int, ...]], n: int = N) -> np.ndarray:
    """Permutation matrix of a permutation given in 1-indexed cyclic notation.

    Reading (the paper does not say whether P acts on positions or values):
    (P x)_i = x_{sigma(i)}, where sigma maps each element of a cycle to the
    next one.  This is the only one of the four conventions (positions or
    values, sigma or its inverse) under which the factor product equals the
    printed T; ``tests/test_oracle_pins.py`` checks that the other three fail.
    """
    sigma = list(range(n))
    for cyc in cycles:
        for k, a in enumerate(cyc):
            b = cyc[(k + 1) % len(cyc)]
            sigma[a - 1] = b - 1
    P = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        P[i, sigma[i]] = 1
    return P


# The permutations of Sec. 2.2 in cyclic notation.  The printed cycles
# "(10 12 16 10)", "(11 13 15 11)" and "(3 8 16 ... 13 3)" repeat their first
# element at the end; read as closing the cycle, i.e. (10 12 16), (11 13 15)
# and (3 8 16 15 5 4 12 11 7 6 10 14 13).
P1_CYCLES = [(10, 12, 16), (11, 13, 15)]
P2_CYCLES = [(2, 9), (3, 8, 16, 15, 5, 4, 12, 11, 7, 6, 10, 14, 13)]


def factor_matrices() -> dict[str, np.ndarray]:
    """The six factors of Sec. 2.2, built from the paper's block descriptions."""
    M1 = _butterfly(16)
    M2 = _block_diag(_butterfly(8), _butterfly(8))
    M3 = _block_diag(_butterfly(4), -_eye(4), _butterfly(4), -_eye(4))
    M4 = _block_diag(
        np.array([[1, 1, 0], [1, -1, 0], [0, 0, -1]], dtype=np.int64),
        _eye(4),
        np.array([[-1, 0, 0], [0, 1, 1], [0, 1, -1]], dtype=np.int64),
        -_eye(4),
        np.array([[1, 0], [0, -1]], dtype=np.int64),
    )
    return {
        "M1": M1,
        "P1": _cycles_to_matrix(P1_CYCLES),
        "M2": M2,
        "M3": M3,
        "M4": M4,
        "P2": _cycles_to_matrix(P2_CYCLES),
    }


# Order in which the factors act on a column vector (rightmost first).
FACTOR_ORDER = ("M1", "P1", "M2", "M3", "M4", "P2")


def stage_additions(M: np.ndarray) -> int:
    """Additions needed to apply a {0,+-1} matrix: per row, (nonzeros - 1).

    Sign changes and permutations cost nothing (Sec. 2.2, Table 1)."""
    nnz = np.count_nonzero(M, axis=1)
    return int(np.sum(np.maximum(nnz - 1, 0)))


def apply_stage(M: np.ndarray, x: np.ndarray, dtype=np.int64) -> np.ndarray:
    """Apply a sparse {0,+-1} stage matrix to the vectors in the LAST axis of x.

    Each output is the signed sum of the inputs its row selects, added left to
    right in ``dtype`` (so, for the two-term rows of the factorisation, one
    rounded addition per output in float32).  Returns (out, additions)."""
    x = np.asarray(x, dtype=dtype)
    out = np.zeros(x.shape, dtype=dtype)
    adds = 0
    for i in range(M.shape[0]):
        cols = np.nonzero(M[i])[0]
        acc = None
        for j in cols:
            term = x[..., j] if M[i, j] > 0 else -x[..., j]
            if acc is None:
                acc = term.astype(dtype)
            else:
                acc = (acc + term).astype(dtype)
                adds += 1
        out[..., i] = acc if acc is not None else 0
    return out, adds


def t16_factored(x: np.ndarray) -> tuple[np.ndarray, int]:
    """y = T x for every 16-vector in the last axis of x, through the factors
    in the paper's order (M1 first, P2 last), exact int64.  Returns (y, adds)
    where adds counts the additions one 16-vector costs."""
    F = factor_matrices()
    y = np.asarray(x, dtype=np.int64)
    total = 0
    for name in FACTOR_ORDER:
        y, a = apply_stage(F[name], y, np.int64)
        total += a
    return y, total


def t16_transpose_factored_fp32(x: np.ndarray) -> np.ndarray:
    """y = T^t x in binary32, through the transposed factorisation
    T^t = M1^t P1^t M2^t M3^t M4^t P2^t, applied stage by stage (P2^t first).

    Every stage row has at most two nonzeros, so each output of each stage is
    one float32 addition of two float32 values: the rounding of the whole
    evaluation is fixed by the factorisation."""
    F = factor_matrices()
    y = np.asarray(x, dtype=np.float32)
    for name in reversed(FACTOR_ORDER):
        y, _ = apply_stage(F[name].T, y, np.float32)
    return y


# ---------------------------------------------------------------------------
# Sec. 3.1: blocks, forward 2-D transform, zig-zag zonal mask, inverse.
# ---------------------------------------------------------------------------
def image_to_blocks(img: np.ndarray) -> np.ndarray:
    """Split an H x W image (H, W multiples of 16) into (H/16)(W/16) disjoint
    16x16 blocks in raster block order; result shape (nblk, 16, 16)."""
    H, W = img.shape
    if H % N or W % N:
        raise ValueError("image sides must be multiples of 16")
    b = img.reshape(H // N, N, W // N, N).transpose(0, 2, 1, 3)
    return b.reshape(-1, N, N)


def blocks_to_image(blocks: np.ndarray, H: int, W: int) -> np.ndarray:
    """Inverse of ``image_to_blocks``: rearrange blocks into an H x W image."""
    b = blocks.reshape(H // N, W // N, N, N).transpose(0, 2, 1, 3)
    return b.reshape(H, W)


def forward_direct(blocks: np.ndarray) -> np.ndarray:
    """Y = T X T^t for each block, by direct int64 matrix products (Sec. 3.1
    forward transform with the unscaled T; S is applied in the quantiser)."""
    X = np.asarray(blocks, dtype=np.int64)
    return np.matmul(np.matmul(T, X), T.T)


def forward_factored(blocks: np.ndarray) -> np.ndarray:
    """Y = T X T^t through the 44-addition factorisation: first every row of X
    (X T^t: the transform of each row), then every column of the result."""
    X = np.asarray(blocks, dtype=np.int64)
    rows, _ = t16_factored(X)  # row i of X -> row i of X T^t
    cols, _ = t16_factored(np.swapaxes(rows, -1, -2))  # columns of X T^t
    return np.swapaxes(cols, -1, -2)


def zigzag_order(n: int = N) -> list[tuple[int, int]]:
    """The zig-zag scan of an n x n block as (u, v) = (row, column).

    Reading: the paper cites a zig-zag sequence without printing it; this is
    the JPEG convention extended to n x n.  Anti-diagonals d = u + v are taken
    in increasing order; on odd d the scan runs from row 0 downward, on even d
    from the bottom row upward.  For n = 8 this is the JPEG table, which the
    tests check against the standard's listing."""
    order = []
    for d in range(2 * n - 1):
        cells = [(u, d - u) for u in range(n) if 0 <= d - u < n]  # u ascending
        if d % 2 == 0:
            cells.reverse()
        order.extend(cells)
    return order


def zonal_mask(r: int, n: int = N) -> np.ndarray:
    """Boolean n x n mask keeping the first r coefficients in zig-zag order
    (Sec. 3.1; the paper uses 1 <= r <= 150, r = 256 keeps everything)."""
    if not 1 <= r <= n * n:
        raise ValueError("r must be in 1..256")
    m = np.zeros((n, n), dtype=bool)
    for (u, v) in zigzag_order(n)[:r]:
        m[u, v] = True
    return m


def round_half_away(x: np.ndarray) -> np.ndarray:
    """Round to nearest, ties away from zero (C ``round``), as float64.

    Reading: the paper does not state its rounding rule.  Evaluated in float64,
    which is exact for every binary32 input."""
    x = np.asarray(x, dtype=np.float64)
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def d_factors() -> np.ndarray:
    """d = 4 s: (1, 1, 2, sqrt2, sqrt2, 1, 2, 2, 1, 2, 2, sqrt2, sqrt2, 2, 2, 2)."""
    return 4.0 * S_DIAG


def quantise(Y: np.ndarray, q: float | None, r: int, precision: str = "fp64") -> np.ndarray:
    """Zonal (and optionally uniform) quantisation of coefficient blocks.

    Sec. 3.1 keeps the first r zig-zag coefficients of B = C_hat A C_hat^t and
    zeroes the rest.  With S merged into the quantiser (Sec. 2.1, last
    paragraph), the orthonormal coefficient is c_uv = s_u s_v Y_uv.

    * q is None (the paper's image experiment, no quantiser): returns the
      coefficients c_uv inside the zone (float64), zero outside.
    * q > 0 (reading: a uniform step in the orthonormal domain, as in the
      paper's video experiment): level_uv = round_half_away(c_uv / q) inside
      the zone, 0 outside; an int64 array.

    ``precision='fp32'`` takes the rounding decision in binary32, as the GPU
    does: f_uv = fl32(s_u s_v / q) and level = round_half_away(fl32(fl32(Y_uv)
    * f_uv)), one rounded product.  ``'fp64'`` computes c_uv / q in float64.
    """
    Y = np.asarray(Y, dtype=np.int64)
    mask = zonal_mask(r)
    ss = np.outer(S_DIAG, S_DIAG)
    if q is None:
        return np.where(mask, ss * Y, 0.0)
    if q <= 0:
        raise ValueError("q must be positive")
    if precision == "fp64":
        lev = round_half_away(ss * Y / q)
    elif precision == "fp32":
        f32 = (ss / q).astype(np.float32)
        prod = Y.astype(np.float32) * f32  # binary32 multiply, rounded once
        lev = round_half_away(prod.astype(np.float32))
    else:
        raise ValueError(precision)
    return np.where(mask, lev, 0).astype(np.int64)


def dequantise(levels: np.ndarray, q: float) -> np.ndarray:
    """Orthonormal-domain coefficients back to the unscaled-T domain for the
    inverse: W_uv = s_u s_v q level_uv (float64), so that X = T^t W T equals
    C_hat^t B_tilde C_hat (Sec. 3.1 inverse with C_hat^t = T^t S)."""
    ss = np.outer(S_DIAG, S_DIAG)
    return ss * q * np.asarray(levels, dtype=np.float64)


def inverse_fp64(W: np.ndarray) -> np.ndarray:
    """X_tilde = T^t W T for each block (float64), Sec. 3.1 inverse."""
    Tf = T.astype(np.float64)
    return np.matmul(np.matmul(Tf.T, np.asarray(W, dtype=np.float64)), Tf)


def inverse_fp32(levels: np.ndarray, q: float) -> np.ndarray:
    """X_tilde = T^t W T in binary32, the precision of the GPU inverse.

    W_uv = fl32(fl32(level_uv) * g_uv) with g_uv = fl32(q s_u s_v); then the
    transposed factorisation runs on every column of W (T^t W), then on every
    row of the result ((T^t W) T), stage by stage in binary32."""
    ss = np.outer(S_DIAG, S_DIAG)
    g32 = (q * ss).astype(np.float32)
    W = np.asarray(levels, dtype=np.int64).astype(np.float32) * g32
    W = W.astype(np.float32)
    cols = t16_transpose_factored_fp32(np.swapaxes(W, -1, -2))  # T^t W, columnwise
    Z = np.swapaxes(cols, -1, -2)
    return t16_transpose_factored_fp32(Z)  # each row of T^t W -> row of X_tilde


def inverse_exact_zonal(Y: np.ndarray, r: int) -> np.ndarray:
    """No-quantiser inverse in exact integers (returns 256 X_tilde, int64).

    With W = S B_tilde S and B_tilde = mask (S Y S):  X_tilde = (1/256) T^t
    (mask . D' Y D') T with D' = 16 S^2 = diag(1,1,4,2,2,1,4,4,1,4,4,2,2,4,4,4),
    an integer numerator (Sec. 2.1 S, Sec. 3.1 inverse)."""
    Dp = np.rint(16.0 * S_DIAG**2).astype(np.int64)
    mask = zonal_mask(r)
    Wn = np.where(mask, np.asarray(Y, dtype=np.int64) * np.outer(Dp, Dp), 0)
    return np.matmul(np.matmul(T.T, Wn), T)


def pixels_from_exact(num256: np.ndarray, bits: int) -> np.ndarray:
    """round_half_away(num / 256), clipped to [0, 2^bits - 1], exact integers."""
    n = np.asarray(num256, dtype=np.int64)
    mag = (np.abs(n) + 128) // 256
    v = np.where(n >= 0, mag, -mag)
    return np.clip(v, 0, (1 << bits) - 1)


def pixels_from_float(X: np.ndarray, bits: int) -> np.ndarray:
    """Reconstruct pixels: clip(round_half_away(X), 0, 2^bits - 1)."""
    return np.clip(round_half_away(X), 0, (1 << bits) - 1).astype(np.int64)


def sse(a: np.ndarray, b: np.ndarray) -> int:
    """Sum of squared differences, exact integer."""
    d = np.asarray(a, dtype=np.int64) - np.asarray(b, dtype=np.int64)
    return int(np.sum(d * d))


def psnr(sse_value: int, H: int, W: int, bits: int) -> float:
    """PSNR = 10 log10(peak^2 H W / SSE), peak = 2^bits - 1; +inf for SSE = 0.

    Reading: the paper uses PSNR (Sec. 3.1, Sec. 3.2) without printing it; this
    is the standard per-image definition."""
    if sse_value == 0:
        return math.inf
    peak = float((1 << bits) - 1)
    return 10.0 * math.log10(peak * peak * H * W / float(sse_value))


def codec_image(img: np.ndarray, q: float | None, r: int, bits: int = 8,
                precision: str = "fp64", forward: str = "direct") -> dict:
    """The whole Sec. 3.1 codec on one image: blocks, Y = T X T^t, zonal
    (+ uniform) quantisation, inverse, rearrangement, SSE and PSNR.

    * q is None: exact-integer zonal path (``inverse_exact_zonal``); levels
      are the masked integer coefficients Y.
    * q > 0, precision 'fp64': float64 throughout (the definition).
    * q > 0, precision 'fp32': rounding decisions in binary32 along the
      factorisation (``quantise(..., 'fp32')`` and ``inverse_fp32``).
    * forward: 'direct' (int64 matrix products, ``forward_direct``) or
      'factored' (the 44-addition factorisation of Sec. 2.2 stage by stage,
      ``forward_factored``); both give the same Y exactly.
    """
    H, W = img.shape
    X = image_to_blocks(np.asarray(img, dtype=np.int64))
    if forward == "direct":
        Y = forward_direct(X)
    elif forward == "factored":
        Y = forward_factored(X)
    else:
        raise ValueError("forward must be 'direct' or 'factored'")
    if q is None:
        levels = np.where(zonal_mask(r), Y, 0)
        rec = pixels_from_exact(inverse_exact_zonal(Y, r), bits)
    else:
        levels = quantise(Y, q, r, precision)
        if precision == "fp64":
            rec = pixels_from_float(inverse_fp64(dequantise(levels, q)), bits)
        else:
            rec = pixels_from_float(inverse_fp32(levels, q).astype(np.float64), bits)
    out = blocks_to_image(rec, H, W)
    e = sse(img, out)
    return {"Y": Y, "levels": levels, "recon": out, "sse": e,
            "psnr": psnr(e, H, W, bits)}


# ---------------------------------------------------------------------------
# Sec. 2.3, Table 2: similarity and coding measures against the exact DCT-II
# under a first-order Markov (AR(1)) model.  The formulas are the standard
# ones of the cited references (the paper names them without printing them).
# ---------------------------------------------------------------------------
def dct_matrix(n: int = N) -> np.ndarray:
    """Exact orthonormal DCT-II matrix C (row k = frequency k)."""
    k = np.arange(n)
    C = np.sqrt(2.0 / n) * np.cos(np.pi * (2 * k[None, :] + 1) * k[:, None] / (2 * n))
    C[0] /= np.sqrt(2.0)
    return C


def ar1_covariance(rho: float, n: int = N) -> np.ndarray:
    """R_ij = rho^|i-j|, the unit-variance first-order Markov covariance."""
    k = np.arange(n)
    return rho ** np.abs(k[:, None] - k[None, :]).astype(np.float64)


def dct_distortion(A: np.ndarray) -> float:
    """d2 = 1 - ||diag(C A^t)||^2 / ||C A^t||_F^2."""
    M = dct_matrix(A.shape[0]) @ A.T
    return float(1.0 - np.sum(np.diag(M) ** 2) / np.sum(M**2))


def total_error_energy(A: np.ndarray) -> float:
    """epsilon = pi ||C - A||_F^2."""
    return float(np.pi * np.sum((dct_matrix(A.shape[0]) - A) ** 2))


def transform_mse(A: np.ndarray, rho: float = 0.95) -> float:
    """MSE = tr((C - A) R (C - A)^t) / N."""
    n = A.shape[0]
    D = dct_matrix(n) - A
    return float(np.trace(D @ ar1_covariance(rho, n) @ D.T) / n)


def coding_gain(A: np.ndarray, rho: float = 0.95) -> float:
    """C_g = 10 log10( mean_i sigma_i^2 / prod_i (sigma_i^2 ||g_i||^2)^(1/N) ),
    sigma_i^2 the diagonal of A R A^t and g_i the i-th basis vector of A^-1."""
    n = A.shape[0]
    RY = A @ ar1_covariance(rho, n) @ A.T
    G = np.linalg.inv(A)
    var = np.diag(RY)
    norms = np.sum(G**2, axis=0)  # squared norm of column i of A^-1
    num = np.mean(var)
    den = np.exp(np.mean(np.log(var * norms)))
    return float(10.0 * np.log10(num / den))


def transform_efficiency(A: np.ndarray, rho: float = 0.95) -> float:
    """eta = 100 sum_i |(A R A^t)_ii| / sum_ij |(A R A^t)_ij|."""
    n = A.shape[0]
    RY = A @ ar1_covariance(rho, n) @ A.T
    return float(100.0 * np.sum(np.abs(np.diag(RY))) / np.sum(np.abs(RY)))


# ---------------------------------------------------------------------------
# Sizes that are not multiples of 16, and colour.
# ---------------------------------------------------------------------------
def pad_to_blocks(img: np.ndarray) -> np.ndarray:
    """Extend an image to the next multiple of 16 in both directions by
    repeating its last row and last column.

    Reading: the paper's images are 512 x 512 and split exactly into 16 x 16
    blocks (Sec. 3.1); for other sizes we take the usual block-codec practice
    of edge replication."""
    H, W = img.shape
    Hp, Wp = -(-H // N) * N, -(-W // N) * N
    return np.pad(np.asarray(img), ((0, Hp - H), (0, Wp - W)), mode="edge")


def codec_image_any_size(img: np.ndarray, q: float | None, r: int, bits: int = 8,
                         precision: str = "fp64") -> dict:
    """The Sec. 3.1 codec on an image of any size: pad by edge replication
    (``pad_to_blocks``), code, keep the original H x W region; SSE and PSNR
    over the original pixels only."""
    H, W = img.shape
    res = codec_image(pad_to_blocks(img), q, r, bits, precision)
    rec = res["recon"][:H, :W]
    e = sse(img, rec)
    return {"recon": rec, "sse": e, "psnr": psnr(e, H, W, bits), "levels": res["levels"]}


def codec_colour(planes: list[np.ndarray], q: float | None, r: int, bits: int = 8,
                 precision: str = "fp64") -> list[dict]:
    """Colour images: each channel coded separately (Sec. 3.1, 'Color images
    could be treated similarly by processing each channel separately')."""
    return [codec_image_any_size(p, q, r, bits, precision) for p in planes]


# ---------------------------------------------------------------------------
# Sec. 3.1, Fig. 2(b) and Fig. 3: SSIM, the paper's second quality measure.
# The paper cites Wang, Bovik, Sheikh and Simoncelli (2004) without fixing the
# window or constants.  Reading: that article's own choices -- an 11 x 11
# circular-symmetric Gaussian window with standard deviation 1.5, normalised
# to unit sum; K1 = 0.01, K2 = 0.03, L = 2^bits - 1; local statistics at every
# position where the window lies wholly inside the image (no padding); no
# downsampling; the mean over those positions (MSSIM).
# ---------------------------------------------------------------------------
SSIM_SIZE = 11
SSIM_SIGMA = 1.5
SSIM_K1 = 0.01
SSIM_K2 = 0.03


def ssim_window(size: int = SSIM_SIZE, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """w(a, b) proportional to exp(-(a^2 + b^2) / (2 sigma^2)), a, b in
    -(size-1)/2 .. (size-1)/2, normalised so that the weights sum to 1."""
    h = (size - 1) // 2
    a = np.arange(-h, h + 1, dtype=np.float64)
    w = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2.0 * sigma * sigma))
    return w / w.sum()


def window_mean(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Weighted local mean at every position where the window fits:
    out[i, j] = sum_{a, b} w[a, b] img[i + a, j + b] (the 2-D window applied
    directly, one shifted copy of the image per weight)."""
    img = np.asarray(img, dtype=np.float64)
    k = w.shape[0]
    H, W = img.shape
    out = np.zeros((H - k + 1, W - k + 1))
    for a in range(k):
        for b in range(k):
            out += w[a, b] * img[a:a + H - k + 1, b:b + W - k + 1]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray, bits: int = 8) -> np.ndarray:
    """Local SSIM (Wang et al. 2004, eq. 13 with the window's weighted
    statistics): ((2 mu_x mu_y + C1)(2 s_xy + C2)) /
    ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)), C1 = (K1 L)^2,
    C2 = (K2 L)^2; s_x^2 = E_w[x^2] - mu_x^2, s_xy = E_w[x y] - mu_x mu_y."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if min(x.shape) < SSIM_SIZE or x.shape != y.shape:
        raise ValueError("SSIM needs two images of equal shape, both sides >= 11")
    L = float((1 << bits) - 1)
    C1 = (SSIM_K1 * L) ** 2
    C2 = (SSIM_K2 * L) ** 2
    w = ssim_window()
    mx, my = window_mean(x, w), window_mean(y, w)
    sxx = window_mean(x * x, w) - mx * mx
    syy = window_mean(y * y, w) - my * my
    sxy = window_mean(x * y, w) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(x: np.ndarray, y: np.ndarray, bits: int = 8) -> float:
    """Mean SSIM over all window positions (MSSIM)."""
    return float(np.mean(ssim_map(x, y, bits)))


# ---------------------------------------------------------------------------
# Sec. 2.1 and Sec. 3.2: the 8-point approximation T8 from which T is built
# (14 additions), the 8x8 block codec it gives, and the mixed tiling of the
# video experiment's second scenario (8- and 16-point transforms together).
# ---------------------------------------------------------------------------
def t8_stages() -> list[tuple[str, np.ndarray]]:
    """The half of the factorisation that acts on the sums a_j = x_j +
    x_{15-j} (the first 8 outputs of M1): M2, M3 and M4 are block diagonal
    across the split of their 16 inputs into 0..7 and 8..15, and their
    top-left 8 x 8 blocks form the 8-point network.  Returned in the order
    they act."""
    F = factor_matrices()
    out = []
    for name in ("M2", "M3", "M4"):
        M = F[name]
        if np.any(M[:8, 8:]) or np.any(M[8:, :8]):
            raise AssertionError(f"{name} is not block diagonal across 8")
        out.append((name, M[:8, :8].copy()))
    return out


def t8_output_order() -> list[int]:
    """g8[k]: the first-half network output that P2 sends to row 2k of T.
    The even rows of T are symmetric (T[2k][j] = T[2k][15-j]), i.e. they see
    only the sums, so they are the 8-point transform in frequency order."""
    P2 = factor_matrices()["P2"]
    g8 = []
    for k in range(8):
        j = int(np.argmax(P2[2 * k]))  # (P2 e)[2k] = e[j]
        if j >= 8:
            raise AssertionError("an even row of T comes from the difference half")
        g8.append(j)
    return g8


def t8_matrix() -> np.ndarray:
    """T8 = rows g8 of M4' M3' M2' (the top-left blocks), an 8 x 8 {0, +-1}
    matrix."""
    G = np.eye(8, dtype=np.int64)
    for _, M in t8_stages():
        G = M @ G
    return G[t8_output_order()]


def t8_factored(x: np.ndarray) -> tuple[np.ndarray, int]:
    """T8 x through the three stages (last axis), int64; returns (y, adds)."""
    y = np.asarray(x, dtype=np.int64)
    adds = 0
    for _, M in t8_stages():
        y, a = apply_stage(M, y)
        adds += a
    return y[..., t8_output_order()], adds


def t8_transpose_factored_fp32(x: np.ndarray) -> np.ndarray:
    """T8^t x in binary32 through the transposed stages: the inputs go to the
    network outputs they came from (g8), then M4'^t, M3'^t, M2'^t, each output
    one rounded addition."""
    x = np.asarray(x, dtype=np.float32)
    y = np.zeros_like(x)
    y[..., t8_output_order()] = x
    for _, M in reversed(t8_stages()):
        y, _ = apply_stage(M.T, y, np.float32)
    return y


def s8_diag() -> np.ndarray:
    """S8 = sqrt((T8 T8^t)^-1), the orthogonalising diagonal of T8 (T8 T8^t
    is diagonal)."""
    G = t8_matrix() @ t8_matrix().T
    if np.any(G - np.diag(np.diag(G))):
        raise AssertionError("T8 T8^t is not diagonal")
    return 1.0 / np.sqrt(np.diag(G).astype(np.float64))


def image_to_blocks8(img: np.ndarray) -> np.ndarray:
    """Disjoint 8 x 8 blocks in raster block order, shape (nblk, 8, 8)."""
    H, W = img.shape
    b = np.asarray(img).reshape(H // 8, 8, W // 8, 8).transpose(0, 2, 1, 3)
    return b.reshape(-1, 8, 8)


def blocks8_to_image(blocks: np.ndarray, H: int, W: int) -> np.ndarray:
    b = np.asarray(blocks).reshape(H // 8, W // 8, 8, 8).transpose(0, 2, 1, 3)
    return b.reshape(H, W)


def forward8(blocks: np.ndarray) -> np.ndarray:
    """Y8 = T8 X T8^t (direct int64 products)."""
    T8 = t8_matrix()
    return np.matmul(np.matmul(T8, np.asarray(blocks, np.int64)), T8.T)


def quantise8(Y: np.ndarray, q: float | None, r: int, precision: str = "fp64") -> np.ndarray:
    """The quantiser of ``quantise`` on 8 x 8 blocks: S8 merged, the first r
    (1..64) zig-zag cells kept; q None keeps s8_u s8_v Y8 inside the zone."""
    Y = np.asarray(Y, dtype=np.int64)
    mask = zonal_mask(r, 8)
    s8 = s8_diag()
    ss = np.outer(s8, s8)
    if q is None:
        return np.where(mask, ss * Y, 0.0)
    if precision == "fp64":
        lev = round_half_away(ss * Y / q)
    else:
        f32 = (ss / q).astype(np.float32)
        lev = round_half_away((Y.astype(np.float32) * f32).astype(np.float32))
    return np.where(mask, lev, 0).astype(np.int64)


def inverse8_fp64(levels: np.ndarray, q: float) -> np.ndarray:
    s8 = s8_diag()
    W = np.outer(s8, s8) * q * np.asarray(levels, np.float64)
    T8 = t8_matrix().astype(np.float64)
    return np.matmul(np.matmul(T8.T, W), T8)


def inverse8_fp32(levels: np.ndarray, q: float) -> np.ndarray:
    """T8^t W T8 in binary32: W = fl32(level * fl32(q s8_u s8_v)), the
    transposed network on the columns of W, then on the rows."""
    s8 = s8_diag()
    g32 = (q * np.outer(s8, s8)).astype(np.float32)
    W = (np.asarray(levels, np.int64).astype(np.float32) * g32).astype(np.float32)
    cols = t8_transpose_factored_fp32(np.swapaxes(W, -1, -2))
    return t8_transpose_factored_fp32(np.swapaxes(cols, -1, -2))


def inverse8_exact_zonal(Y: np.ndarray, r: int) -> np.ndarray:
    """No quantiser: 64 X_tilde = T8^t (mask . D8 Y D8) T8 with D8 = 8 S8^2
    (integers), returned as int64 numerators."""
    D8 = np.rint(8.0 * s8_diag() ** 2).astype(np.int64)
    Wn = np.where(zonal_mask(r, 8), np.asarray(Y, np.int64) * np.outer(D8, D8), 0)
    T8 = t8_matrix()
    return np.matmul(np.matmul(T8.T, Wn), T8)


def pixels_from_exact64(num64: np.ndarray, bits: int) -> np.ndarray:
    """round_half_away(num / 64), clipped, exact integers."""
    n = np.asarray(num64, dtype=np.int64)
    mag = (np.abs(n) + 32) // 64
    return np.clip(np.where(n >= 0, mag, -mag), 0, (1 << bits) - 1)


def codec_blocks8(blocks: np.ndarray, q: float | None, r: int, bits: int = 8,
                  precision: str = "fp64") -> np.ndarray:
    """The Sec. 3.1 codec on 8 x 8 blocks with T8: reconstructed samples."""
    Y = forward8(blocks)
    if q is None:
        return pixels_from_exact64(inverse8_exact_zonal(Y, r), bits)
    lev = quantise8(Y, q, r, precision)
    X = inverse8_fp64(lev, q) if precision == "fp64" else inverse8_fp32(lev, q).astype(np.float64)
    return pixels_from_float(X, bits)


def codec_image_mixed(img: np.ndarray, q: float | None, r16: int, r8: int, bits: int = 8,
                      mode: str = "auto", precision: str = "fp64") -> dict:
    """Mixed 8/16 tiling (the video experiment's second scenario, Sec. 3.2):
    every 16 x 16 region is coded either as one block with T or as four 8 x 8
    blocks with T8.  Reading: the paper leaves the choice to the encoder (HM's
    rate-distortion search); here it is the tiling with the smaller squared
    error of the region, ties to 16 x 16 ('auto'), or forced ('16', '8').
    Returns recon, the split map (one flag per region), SSE and PSNR."""
    H, W = img.shape
    x = np.asarray(img, dtype=np.int64)
    rec16 = codec_image(x, q, r16, bits, precision)["recon"]
    rec8 = blocks8_to_image(codec_blocks8(image_to_blocks8(x), q, r8, bits, precision), H, W)
    d16 = (x - rec16) ** 2
    d8 = (x - rec8) ** 2
    e16 = d16.reshape(H // 16, 16, W // 16, 16).sum(axis=(1, 3))
    e8 = d8.reshape(H // 16, 16, W // 16, 16).sum(axis=(1, 3))
    if mode == "auto":
        split = e8 < e16
    elif mode == "16":
        split = np.zeros_like(e16, dtype=bool)
    elif mode == "8":
        split = np.ones_like(e16, dtype=bool)
    else:
        raise ValueError(mode)
    sel = np.kron(split, np.ones((16, 16), dtype=bool))
    rec = np.where(sel, rec8, rec16)
    e = sse(x, rec)
    return {"recon": rec, "split": split, "sse": e, "psnr": psnr(e, H, W, bits)}
