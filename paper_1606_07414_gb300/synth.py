"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on 512x512 8-bit natural images and CIF video; neither is
available here, so the inputs are first-order Markov (AR(1)) Gaussian fields,
the model the paper names for natural images (Sec. 1, and rho = 0.95 in
Table 2), rounded and clipped to the sample range.

This module holds random numbers and field synthesis only -- none of the
transform, quantiser or PSNR arithmetic -- so that both the CUDA path's tests
and the CPU oracle can consume the same bytes.

Random stream: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used counter-style -- output k of seed s is
mix(s + (k + 1) * 0x9E3779B97F4A7C15) -- mapped to doubles by the top 53 bits,
then to normals by the Box-Muller transform.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream of ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in (0, 1]: ((x >> 11) + 1) * 2^-53."""
    x = splitmix64(seed, count, offset)
    return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive pairs of uniforms."""
    m = (count + 1) // 2
    u = uniforms(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def _ar1_along(z: np.ndarray, rho: float, axis: int) -> np.ndarray:
    """f[0] = z[0], f[k] = rho f[k-1] + sqrt(1 - rho^2) z[k] along ``axis``:
    a stationary unit-variance AR(1) sequence."""
    from scipy.signal import lfilter

    b = np.sqrt(1.0 - rho * rho)
    zz = np.moveaxis(z, axis, -1).copy()
    zz[..., 0] /= b  # so that f[0] = b * (z[0] / b) = z[0]
    f = lfilter([b], [1.0, -rho], zz, axis=-1)
    return np.moveaxis(f, -1, axis)


def ar1_field(seed: int, H: int, W: int, rho: float) -> np.ndarray:
    """A separable AR(1) Gaussian field, unit variance, correlation
    rho^|di| rho^|dj|: filtered along rows, then along columns."""
    z = normals(seed, H * W).reshape(H, W)
    return np.ascontiguousarray(_ar1_along(_ar1_along(z, rho, axis=1), rho, axis=0))


def to_samples(field: np.ndarray, bits: int, mean: float | None = None,
               std: float | None = None) -> np.ndarray:
    """clip(round_half_away(mean + std * field), 0, 2^bits - 1).

    Defaults: mean 128 / std 50 for 8-bit, scaled by 2^(bits-8) otherwise
    (mean 512 / std 200 for 10-bit)."""
    scale = float(1 << (bits - 8))
    mean = 128.0 * scale if mean is None else mean
    std = 50.0 * scale if std is None else std
    v = mean + std * field
    v = np.sign(v) * np.floor(np.abs(v) + 0.5)
    v = np.clip(v, 0, (1 << bits) - 1)
    return np.ascontiguousarray(v.astype(np.uint8 if bits == 8 else np.uint16))


def ar1_image(seed: int, H: int, W: int, rho: float = 0.95, bits: int = 8) -> np.ndarray:
    """One H x W sample image (uint8 for 8 bits, uint16 otherwise)."""
    return to_samples(ar1_field(seed, H, W, rho), bits)


def image_batch(seed: int, n: int, H: int, W: int, rho_lo: float, rho_hi: float,
                bits: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """n images of H x W; image i has seed ``seed + i`` and rho drawn
    uniformly in [rho_lo, rho_hi] from the stream of ``seed``.
    Returns (images (n, H, W), rhos (n,))."""
    rhos = rho_lo + (rho_hi - rho_lo) * uniforms(seed ^ 0x5EED, n)
    imgs = np.empty((n, H, W), dtype=np.uint8 if bits == 8 else np.uint16)
    for i in range(n):
        imgs[i] = ar1_image(seed + 1 + i, H, W, float(rhos[i]), bits)
    return imgs, rhos


def video_frames(seed: int, n: int, H: int = 1088, W: int = 1920, rho: float = 0.95,
                 step: int = 2, margin: int = 32, bits: int = 8) -> np.ndarray:
    """n frames cropped from one AR(1) field with a random walk of offsets:
    frame k's offset moves by (dx, dy), each uniform in {-step..step}, and is
    clamped to a margin of ``margin`` pixels around the frame (a stand-in for
    the camera motion of video).  Returns (n, H, W)."""
    base = ar1_image(seed, H + 2 * margin, W + 2 * margin, rho, bits)
    u = uniforms(seed ^ 0xF4A3E5, 2 * n)
    steps = np.minimum(np.floor(u * (2 * step + 1)), 2 * step).astype(np.int64) - step
    out = np.empty((n, H, W), dtype=base.dtype)
    oy = ox = 0
    for k in range(n):
        if k > 0:
            oy = int(np.clip(oy + steps[2 * k], -margin, margin))
            ox = int(np.clip(ox + steps[2 * k + 1], -margin, margin))
        out[k] = base[margin + oy: margin + oy + H, margin + ox: margin + ox + W]
    return out


def uneven_sizes(seed: int, n: int, lo: int = 64, hi: int = 4096, mult: int = 16
                 ) -> tuple[np.ndarray, np.ndarray]:
    """n (H, W) pairs, each side uniform over the multiples of ``mult`` in
    [lo, hi], independently."""
    k = (hi - lo) // mult + 1
    u = uniforms(seed ^ 0x512E5, 2 * n)
    idx = np.minimum(np.floor(u * k), k - 1).astype(np.int64)
    return lo + mult * idx[0::2], lo + mult * idx[1::2]


def choice(seed: int, n: int, values) -> np.ndarray:
    """n draws, uniform over ``values``."""
    values = np.asarray(values)
    u = uniforms(seed, n)
    return values[np.minimum(np.floor(u * len(values)), len(values) - 1).astype(np.int64)]
