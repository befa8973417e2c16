"""CPU checks of the binary32 identities the fused kernels rely on, with
directed rounding emulated exactly: a binary32 operation on binary32 inputs
is computed exactly in float64 (enough bits for every case here) and then
rounded down to binary32 by hand.

  * sample rounding: the bits of RD(RD(X + 1/2) * 2^-149), read as int32 and
    clamped to [0, peak], equal clip(floor(X + 1/2), 0, peak) -- the exact
    rounding of a reconstructed sample (half away from zero; negatives clip
    to 0 either way);
  * level magnitude: RD(RD(|t| + 1/2) + 2^23) - 2^23 = floor(|t| + 1/2) for
    |t| + 1/2 < 2^23.
"""
import numpy as np

F32 = np.float32


def rd32(exact):
    """Round float64 values (exact results) down to binary32."""
    f = exact.astype(F32)  # to nearest, subnormals included
    over = f.astype(np.float64) > exact
    return np.where(over, np.nextafter(f, F32(-np.inf)), f)


def sample_bits(x32, peak):
    v = rd32(x32.astype(np.float64) + 0.5)
    n = rd32(v.astype(np.float64) * 2.0 ** -149)  # exact product, then down to the subnormal grid
    return np.clip(n.view(np.int32).astype(np.int64), 0, peak)


def _cases():
    rng = np.random.default_rng(1606)
    k = np.arange(-20, 4200, dtype=np.float64)
    ties = (k + 0.5).astype(F32)
    xs = [rng.uniform(-600, 4700, 400_000).astype(F32), ties,
          np.nextafter(ties, F32(-np.inf)), np.nextafter(ties, F32(np.inf)),
          k.astype(F32), np.nextafter(k.astype(F32), F32(-np.inf)),
          np.array([-0.0, 0.0, -0.5, 0.5, -1e-30, 1e-30, 255.5, 1023.5, 4095.5, 2.0 ** 22, 2.0 ** 23,
                    2.0 ** 24, 1e9, -1e9, 3e38, -3e38], dtype=F32)]
    return np.concatenate(xs)


def test_sample_rounding_through_a_subnormal():
    x = _cases()
    for bits in (8, 10, 12):
        peak = (1 << bits) - 1
        want = np.clip(np.floor(x.astype(np.float64) + 0.5), 0, peak).astype(np.int64)
        assert np.array_equal(sample_bits(x, peak), want), bits


def test_rd_then_floor_keeps_the_floor():
    """floor(RD(v)) = floor(v): the integer below v is a binary32 value not above v."""
    x = _cases()
    x = x[np.abs(x) < 2.0 ** 24]
    v = x.astype(np.float64) + 0.5
    assert np.array_equal(np.floor(rd32(v).astype(np.float64)), np.floor(v))


def test_level_magnitude_by_the_2_23_shift():
    rng = np.random.default_rng(7)
    a = np.abs(np.concatenate([rng.uniform(0, 2.0 ** 22, 300_000), np.arange(0, 5000) + 0.5,
                               np.arange(0, 5000) + 0.4999999, [0.0, 2.0 ** 23 - 1.0]])).astype(F32)
    m = rd32(rd32(a.astype(np.float64) + 0.5).astype(np.float64) + 2.0 ** 23)
    got = m.astype(np.float64) - 2.0 ** 23
    assert np.array_equal(got, np.floor(a.astype(np.float64) + 0.5))


def test_t8_lower_blocks_run_bottom_up():
    """The mixed-tiling kernel runs the lower 8x8 blocks bottom-up in the
    second lane (row 7 - i beside row i of the upper block), so both lanes use
    the same T8 networks.  That rests on two identities, checked here on the
    oracle's own T8 and its binary32 transposed network:
      * forward: T8 applied to a reversed column gives (-1)^u times T8 of the
        column (row u of T8 is symmetric for even u, antisymmetric for odd u);
      * inverse: the binary32 transposed network applied to (-1)^u w gives the
        reversed result of applying it to w, bit for bit (each stage output is
        one rounded operation, and rounding to nearest is odd-symmetric)."""
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import tx16_oracle as O

    T8 = O.t8_matrix()
    sign = np.array([(-1) ** u for u in range(8)], dtype=np.int64)
    rng = np.random.default_rng(8)
    cols = rng.integers(-40000, 40000, size=(2000, 8))
    assert np.array_equal(cols[:, ::-1] @ T8.T, (cols @ T8.T) * sign)
    # binary32 inverse on random coefficients, with exact zeros and ties of magnitude
    w = (rng.standard_normal((4000, 8)) * rng.choice([1.0, 100.0, 1e4], size=(4000, 1))).astype(F32)
    w[::7, 3:] = 0.0
    z = O.t8_transpose_factored_fp32(w)
    zs = O.t8_transpose_factored_fp32((w * sign.astype(F32)).astype(F32))
    assert np.array_equal(zs.view(np.int32), z[:, ::-1].view(np.int32))
