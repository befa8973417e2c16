// Pieces shared by the two fused 8-bit codec kernels (tx16_fused.cu: two
// blocks per thread pair through shared memory; tx16_fused_bt.cu: one block
// per thread in registers): the zonal classes with their pruned networks, the
// exact byte-to-float and float-to-binary16 conversions, block coordinates
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
using ZoneD = Zone<11, 10, FwdRow10, FwdCol11, InvCol11, InvRow10, 5>;  // r <= 64
using ZoneE = Zone<16, 16, FwdRow16, FwdCol16, InvCol16, InvRow16, 4>;  // any r

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// 2^23 + byte k of w, as a float (exact)
__device__ __forceinline__ float biased(unsigned w, int k) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u | unsigned(k)));
}

// fl32 pair -> f16 pair with round toward zero; .x goes to the low half
__device__ __forceinline__ unsigned cvt_rz_h2(float2 v) {
  unsigned d;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.y), "f"(v.x));
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
