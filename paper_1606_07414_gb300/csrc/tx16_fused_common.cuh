// Pieces shared by the two fused 8-bit codec kernels (tx16_fused.cu: two
// blocks per thread pair through shared memory; tx16_fused_bt.cu: one block
// per thread in registers): the zonal classes with their pruned networks, the
// exact byte-to-float conversion and sample rounding, block coordinates
// and the per-image SSE flush.
#pragma once

#include <cuda_runtime.h>

#include "tx16_internal.h"
#include "tx16_pairnet.cuh"

namespace tx16 {
namespace {

using namespace pairnet;

template <int U_, int V_, class FR, class FC, class IC, class IR, int MINB>
struct Zone {
  static constexpr int U = U_;  // kept rows u < U
  static constexpr int V = V_;  // kept columns v < V
  static constexpr int kMinCtas = MINB;  // resident CTAs per SM the registers are budgeted for
  using FwdRow = FR;
  using FwdCol = FC;
  using InvCol = IC;
  using InvRow = IR;
};
using ZoneA = Zone<3, 4, FwdRow4, FwdCol3, InvCol3, InvRow4, 8>;        // r <= 8
using ZoneB = Zone<5, 6, FwdRow6, FwdCol5, InvCol5, InvRow6, 8>;        // r <= 16
using ZoneC = Zone<7, 8, FwdRow8, FwdCol7, InvCol7, InvRow8, 6>;        // r <= 32
// resident CTAs per SM the pair kernel's registers are budgeted for, classes D and E
// (compile-time tunable; measured on 1920x1088 frames: 7 and 6 beat 5 and 4
// by 2.5 and 5 %; more spill)
#ifndef TX16_PAIR_MINCTAS_D
#define TX16_PAIR_MINCTAS_D 7
#endif
#ifndef TX16_PAIR_MINCTAS_E
#define TX16_PAIR_MINCTAS_E 6
#endif
using ZoneD = Zone<11, 10, FwdRow10, FwdCol11, InvCol11, InvRow10, TX16_PAIR_MINCTAS_D>;  // r <= 64
using ZoneE = Zone<16, 16, FwdRow16, FwdCol16, InvCol16, InvRow16, TX16_PAIR_MINCTAS_E>;  // any r

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// 2^23 + byte k of w, as a float (exact)
__device__ __forceinline__ float biased(unsigned w, int k) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | unsigned(k)));
}

// Exact rounding of reconstructed samples, clip(floor(X + 1/2), 0, peak), in
// two packed operations and a saturating pack:
//   v = RD(X + 1/2)     floor(v) = floor(X + 1/2): that integer is a binary32
//                       value not above X + 1/2, so RD cannot fall below it;
//   RD(v * 2^-149)      the multiple of the smallest subnormal not above
//                       v * 2^-149: for 0 <= v < 2^23 the subnormal whose bits
//                       are the integer floor(v); for v < 0 a negative value
//                       (or -0), whose bits read as int32 are negative; for
//                       larger v a value whose bits exceed any peak (the bits
//                       of non-negative floats are ordered like their values).
// The bits, read as int32, are then clamped to [0, peak] as integers.
// (The flush of subnormals is off in this build: no -ftz, no fast math.)
__device__ __forceinline__ float2 floor_bits2(float2 v) { return __fmul2_rd(v, f2(__int_as_float(1))); }

// four int32 values clamped to [0, 255], as the bytes s0 (lowest) .. s3 of one word
__device__ __forceinline__ unsigned pack4_sat_u8(int s0, int s1, int s2, int s3) {
  unsigned t, d;
  // cvt.pack.sat.u8.s32.b32 d, a, b, c: d = c << 16 | sat(a) << 8 | sat(b)
  asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(t) : "r"(s3), "r"(s2), "r"(0));
  asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(s1), "r"(s0), "r"(t));
  return d;
}

// two int32 values clamped to [0, peak] (peak < 2^16), as the low (s0) and
// high (s1) halves of one word: saturating pack to [0, 65535], then a packed
// 16-bit minimum with the peak
__device__ __forceinline__ unsigned pack2_sat_u16(int s0, int s1, unsigned peak2) {
  unsigned t, d;
  // cvt.pack.sat.u16.s32 d, a, b: d = sat(a) << 16 | sat(b)
  asm("cvt.pack.sat.u16.s32 %0, %1, %2;" : "=r"(t) : "r"(s1), "r"(s0));
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(t), "r"(peak2));
  return d;
}

// (by, bx) of block blk: umulhi quotient, exact or one short, then corrected
__device__ __forceinline__ int2 block_coords(unsigned magic, int nbx, int blk) {
  int q = int(__umulhi(unsigned(blk), magic));
  int r = blk - q * nbx;
  const bool over = r >= nbx;
  q += over ? 1 : 0;
  r -= over ? nbx : 0;
  return make_int2(q, r);
}

__device__ __forceinline__ void flush_sse(unsigned long long* sse, int img, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicAdd(sse + img, v);
}

// The image whose tile range holds tile t (binary search; tile0 ascending).
__device__ __forceinline__ int image_of_tile(const ImgParam* imgs, int nimg, int t) {
  int lo = 0, hi = nimg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (imgs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace
}  // namespace tx16
