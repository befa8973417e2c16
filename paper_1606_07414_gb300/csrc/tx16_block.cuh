// Device helpers of the general (16 threads per block, int32) kernels:
// 16-sample row I/O for 8- and 16-bit planes, exact rounding, the per-image
// SSE flush, and the inverse of one block from its column-held coefficients.
#pragma once

#include <cuda_runtime.h>

#include "tx16_internal.h"
#include "tx16_net.cuh"

namespace tx16 {

// ---------------------------------------------------------------------------
// Sample rows: 16 samples = 16 bytes (uint8) or 32 bytes (uint16).
// ---------------------------------------------------------------------------
template <typename Smp>
struct RowIO;

template <>
struct RowIO<uint8_t> {
  static constexpr int kVec = 1;
  __device__ static __forceinline__ void load(const void* p, uint4 (&w)[kVec]) {
    w[0] = __ldcs(reinterpret_cast<const uint4*>(p));
  }
  __device__ static __forceinline__ void unpack(const uint4 (&w)[kVec], int (&x)[16]) {
    const unsigned u[4] = {w[0].x, w[0].y, w[0].z, w[0].w};
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (u[k >> 2] >> (8 * (k & 3))) & 0xffu;
  }
  __device__ static __forceinline__ void store(void* p, const int (&x)[16]) {
    unsigned u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      u[k] = unsigned(x[4 * k]) | (unsigned(x[4 * k + 1]) << 8) | (unsigned(x[4 * k + 2]) << 16) |
             (unsigned(x[4 * k + 3]) << 24);
    __stcs(reinterpret_cast<uint4*>(p), make_uint4(u[0], u[1], u[2], u[3]));
  }
};

template <>
struct RowIO<uint16_t> {
  static constexpr int kVec = 2;
  __device__ static __forceinline__ void load(const void* p, uint4 (&w)[kVec]) {
    w[0] = __ldcs(reinterpret_cast<const uint4*>(p));
    w[1] = __ldcs(reinterpret_cast<const uint4*>(p) + 1);
  }
  __device__ static __forceinline__ void unpack(const uint4 (&w)[kVec], int (&x)[16]) {
    const unsigned u[8] = {w[0].x, w[0].y, w[0].z, w[0].w, w[1].x, w[1].y, w[1].z, w[1].w};
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (u[k >> 1] >> (16 * (k & 1))) & 0xffffu;
  }
  __device__ static __forceinline__ void store(void* p, const int (&x)[16]) {
    unsigned u[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) u[k] = unsigned(x[2 * k]) | (unsigned(x[2 * k + 1]) << 16);
    __stcs(reinterpret_cast<uint4*>(p), make_uint4(u[0], u[1], u[2], u[3]));
    __stcs(reinterpret_cast<uint4*>(p) + 1, make_uint4(u[4], u[5], u[6], u[7]));
  }
};

// (by, bx) of block blk of an image nbx blocks wide, without a division: the
// high product of blk and magic = floor(2^32 / nbx) (2^32 - 1 for nbx = 1) is
// the quotient or one short of it for blk < 2^31, and one compare corrects it
__device__ __forceinline__ void block_row_col(uint32_t magic, int nbx, int blk, int& by, int& bx) {
  int q = int(__umulhi(unsigned(blk), magic));
  int r = blk - q * nbx;
  if (r >= nbx) {
    ++q;
    r -= nbx;
  }
  by = q;
  bx = r;
}

__device__ __forceinline__ int round_div256(int n) {
  // round_half_away(n / 256) in exact integers
  return n >= 0 ? (n + 128) >> 8 : -((128 - n) >> 8);
}

__device__ __forceinline__ void flush_sse_rows(unsigned long long* sse, int img, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicAdd(sse + img, v);
}

// Inverse of one block from the column-held dequantised coefficients
// (thread l holds column v = l of W, rows 0..15) to reconstructed samples of
// row l.  S is this block's 16 x 17 exchange buffer.
template <bool kQuant>
__device__ __forceinline__ void inverse_to_row(int (*S)[17], const int l, const int (&lev)[16],
                                               const ImgParam& I, int (&p)[16]) {
  const int v = l;
  const int ev = scale_class(v);
  const int peak = (1 << (I.flags & 0xff)) - 1;
  if (kQuant) {
    const float g0 = I.g[ev], g1 = I.g[ev + 1], g2 = I.g[ev + 2];
    float w[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int eu = scale_class(u);
      const float gg = eu == 0 ? g0 : (eu == 1 ? g1 : g2);
      w[u] = __fmul_rn(__int2float_rn(lev[u]), gg);
    }
    inv16(w);  // w[i] = (T^t W)[i][v]
#pragma unroll
    for (int i = 0; i < 16; ++i) S[i][v] = __float_as_int(w[i]);
    __syncwarp();
    float z[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) z[j] = __int_as_float(S[l][j]);
    inv16(z);  // row l of X_tilde = (T^t W) T
#pragma unroll
    for (int j = 0; j < 16; ++j) p[j] = int(fminf(fmaxf(roundf(z[j]), 0.f), float(peak)));
  } else {
    int w[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) w[u] = lev[u] * (1 << (scale_class(u) + ev));  // D'_u Y D'_v
    inv16(w);
#pragma unroll
    for (int i = 0; i < 16; ++i) S[i][v] = w[i];
    __syncwarp();
    int z[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) z[j] = S[l][j];
    inv16(z);  // 256 X_tilde, exact
#pragma unroll
    for (int j = 0; j < 16; ++j) p[j] = min(max(round_div256(z[j]), 0), peak);
  }
}

}  // namespace tx16
