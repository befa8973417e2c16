// Fused codec, one 16x16 block per thread, entirely in registers (no level
// output), for 8-bit planes and for 9..12-bit planes in uint16: the kernels,
// templated on the zonal class.
//
// Mapping.  A warp codes a tile of 32 consecutive blocks of one image, lane l
// block 32 t + l, so each 16-byte row load of a warp reads 32 horizontally
// adjacent blocks: 512 contiguous bytes.  Warps take tiles grid-stride, or
// claim them from a work list.
//   row pass     rows i and 15 - i of the block in the two lanes of a float2
//                (i = 0..7): forward row network to the V kept columns, then
//                the column pass's first butterfly (M1 pairs rows i and
//                15 - i) as scalar additions across the lanes, written as
//                column pairs (column 2c, column 2c + 1)
//   column pass  per column pair: the rest of the forward column network,
//                the S-merged quantiser, the inverse column network whose
//                last butterfly (M1 again) writes (row i, row 15 - i) pairs
//   row pass     per row pair: inverse row network, rounding, 16-byte
//                stores of rows i and 15 - i, squared error
// No register moves between the passes, no shared-memory exchange and no
// barrier.  Shared memory holds each thread's 16 input rows (cp.async, one
// stage: refilled with the warp's next tile once the current rows are used,
// the other warps of the SM covering that latency), the column pairs parked
// there to save registers (their column-pass inputs, then in the same slots
// their inverse results), and a small per-warp table of the quantiser
// constants of the image being coded.  The squared error reads the staged
// rows again.
//
// Exactness.  Samples enter as 2^23 + 256 x: every node of the forward
// transform is a multiple of 256 below 2^32 in magnitude (exact in binary32),
// so M1 needs no bias correction; the column pass yields 256 (T X T^t) plus
// 2^31 at (0, 0), removed exactly, and the 1/256 is folded into the
// quantiser's scale.  The quantiser and the inverse follow the library's
// binary32 definition (each stage output one rounded operation on two stage
// inputs, the same as the two-blocks-per-pair kernel in tx16_fused.cu), and
// the sample rounding is exact.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <utility>

#include "tx16_fused_common.cuh"
#include "tx16_internal.h"
#include "tx16_net.cuh"
#include "tx16_pairnet.cuh"

namespace tx16 {
namespace {

constexpr int kWarpTile = 32;  // blocks per warp tile

// Zonal classes of this kernel.  Class c holds the images whose zone lies in
// Z_rmax(c) (zig-zag zones nest: Z_r is a prefix of Z_r' for r <= r').  Per
// class: the kept columns V, the kept rows U, and per column pair the kept
// rows of its taller column, H[cp] (the column heights of Z_rmax); the
// networks are pruned to these at compile time and the per-image scale table
// zeroes what an image's own zone drops.
//   class   A (0)  B (1)   C (2)    D (3)       E (4)                   F (5)
//   r_max   8      16      32       64          128                     256
//   V x U   4 x 3  6 x 5   8 x 7    10 x 11     16 x 15                 16 x 16
//   H       3 2    5 3 1   7 5 4 2  11 9 7 5 3  15 13 11 9 8 6 4 2      16 (x 8)
template <int C>
struct BtClass;
template <>
struct BtClass<0> {
  static constexpr int kRmax = 8, V = 4, U = 3;
  static constexpr int H[2] = {3, 2};
};
template <>
struct BtClass<1> {
  static constexpr int kRmax = 16, V = 6, U = 5;
  static constexpr int H[3] = {5, 3, 1};
};
template <>
struct BtClass<2> {
  static constexpr int kRmax = 32, V = 8, U = 7;
  static constexpr int H[4] = {7, 5, 4, 2};
};
template <>
struct BtClass<3> {
  static constexpr int kRmax = 64, V = 10, U = 11;
  static constexpr int H[5] = {11, 9, 7, 5, 3};
};
template <>
struct BtClass<4> {
  static constexpr int kRmax = 128, V = 16, U = 15;
  static constexpr int H[8] = {15, 13, 11, 9, 8, 6, 4, 2};
};
template <>
struct BtClass<5> {
  static constexpr int kRmax = 256, V = 16, U = 16;
  static constexpr int H[8] = {16, 16, 16, 16, 16, 16, 16, 16};
};
constexpr int kBtClasses = 6;

// The row-pass networks of V kept columns.
template <int V>
struct RowNets;
template <>
struct RowNets<4> {
  using FR = FwdRowT4;
  using IR = InvRow4;
};
template <>
struct RowNets<6> {
  using FR = FwdRowT6;
  using IR = InvRow6;
};
template <>
struct RowNets<8> {
  using FR = FwdRowT8;
  using IR = InvRow8;
};
template <>
struct RowNets<10> {
  using FR = FwdRowT10;
  using IR = InvRow10;
};
template <>
struct RowNets<16> {
  using FR = FwdRowT16;
  using IR = InvRow16;
};

// Per class (compile-time tunable): warps per CTA, resident CTAs per SM the
// registers are budgeted for (the limit per thread is 65536 / (32 * warps *
// CTAs): at most 8 warps per SM allow 255 registers, 9..12 allow 168, 13..16
// allow 128), column pairs parked in shared memory, input stages.  Measured
// on 1920x1088 frames with one input stage (the next tile's rows are fetched
// as the current ones are used; other warps cover the latency) and each warp
// on a contiguous run of tiles (Mblocks/s):
//   A  4-warp CTAs x 3, none parked: 11318 (1-warp x 12: 10901; 4 x 4 with
//      one parked, 16 warps at 128 registers: 10482)
//   B  4-warp CTAs x 3, none parked: 11152 (3 x 4: 11128; 1 x 12: 10983;
//      6 x 2: 10249; 1 x 16 with one parked: 10431)
//   C  4-warp CTAs x 3, one parked: 9729 (none: 9608; two: 9440; 1 x 12 with
//      one: 9683)
//   D  4-warp CTAs x 3, one parked: 7633 (1 x 12 with one: 7514-7522; with
//      two: 7354; 1 x 8 none, 255 registers: 6882)
//   E  1-warp CTAs x 8 (255 registers), two parked: 5482-5539 (three 5357,
//      one 5524; 2-warp x 4: 5381; 4-warp x 2: 5412)
//   F  1-warp CTAs x 8, one parked: 4334-4359 (two 4229, three 4027; 4-warp
//      x 2: 4163)
// Fewer warps with nothing parked beat 16 warps with a pair parked once the
// warps stopped refilling their tables at every tile.
#ifndef TX16_BT_WARPS_A
#define TX16_BT_WARPS_A 4
#endif
#ifndef TX16_BT_MINCTAS_A
#define TX16_BT_MINCTAS_A 3
#endif
#ifndef TX16_BT_PARK_A
#define TX16_BT_PARK_A 0
#endif
#ifndef TX16_BT_WARPS_B
#define TX16_BT_WARPS_B 4
#endif
#ifndef TX16_BT_MINCTAS_B
#define TX16_BT_MINCTAS_B 3
#endif
#ifndef TX16_BT_PARK_B
#define TX16_BT_PARK_B 0
#endif
#ifndef TX16_BT_WARPS_C
#define TX16_BT_WARPS_C 4
#endif
#ifndef TX16_BT_MINCTAS_C
#define TX16_BT_MINCTAS_C 3
#endif
#ifndef TX16_BT_PARK_C
#define TX16_BT_PARK_C 1
#endif
#ifndef TX16_BT_WARPS_D
#define TX16_BT_WARPS_D 4
#endif
#ifndef TX16_BT_MINCTAS_D
#define TX16_BT_MINCTAS_D 3
#endif
#ifndef TX16_BT_PARK_D
#define TX16_BT_PARK_D 1
#endif
#ifndef TX16_BT_WARPS_E
#define TX16_BT_WARPS_E 1
#endif
#ifndef TX16_BT_MINCTAS_E
#define TX16_BT_MINCTAS_E 8
#endif
#ifndef TX16_BT_PARK_E
#define TX16_BT_PARK_E 2
#endif
#ifndef TX16_BT_WARPS_F
#define TX16_BT_WARPS_F 1
#endif
#ifndef TX16_BT_MINCTAS_F
#define TX16_BT_MINCTAS_F 8
#endif
#ifndef TX16_BT_PARK_F
#define TX16_BT_PARK_F 1
#endif
#ifndef TX16_BT_STAGES
#define TX16_BT_STAGES 1
#endif
template <int C>
struct BtLimits;
template <>
struct BtLimits<0> {
  static constexpr int kWarps = TX16_BT_WARPS_A, kMinCtas = TX16_BT_MINCTAS_A, kPark = TX16_BT_PARK_A;
};
template <>
struct BtLimits<1> {
  static constexpr int kWarps = TX16_BT_WARPS_B, kMinCtas = TX16_BT_MINCTAS_B, kPark = TX16_BT_PARK_B;
};
template <>
struct BtLimits<2> {
  static constexpr int kWarps = TX16_BT_WARPS_C, kMinCtas = TX16_BT_MINCTAS_C, kPark = TX16_BT_PARK_C;
};
template <>
struct BtLimits<3> {
  static constexpr int kWarps = TX16_BT_WARPS_D, kMinCtas = TX16_BT_MINCTAS_D, kPark = TX16_BT_PARK_D;
};
template <>
struct BtLimits<4> {
  static constexpr int kWarps = TX16_BT_WARPS_E, kMinCtas = TX16_BT_MINCTAS_E, kPark = TX16_BT_PARK_E;
};
template <>
struct BtLimits<5> {
  static constexpr int kWarps = TX16_BT_WARPS_F, kMinCtas = TX16_BT_MINCTAS_F, kPark = TX16_BT_PARK_F;
};

// Quantiser constants of one image for column pairs c < NP; lane .x is
// column 2c, lane .y column 2c + 1.  The scale is zero outside the zone, so a
// dropped coefficient quantises to level 0 and dequantises to (signed) zero
// with no test of the zone in the kernel body; g depends only on the scale
// classes e(u) = 0, 1, 2.
template <int U, int NP>
struct PairConsts {
  float2 fs[U][NP];  // sign_u f / 256 (quantiser) or sign_u D'_u D'_v / 2^16 (none); 0 outside the zone
  float2 gg[3][NP];  // g
  float2 gc[3][NP];  // -2^23 g
};

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros and
// reads nothing.  The "memory" clobber keeps the compiler from moving shared
// loads of the buffer being refilled across it.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// wait_group with a count known after unrolling (0..7)
__device__ __forceinline__ void cp_async_wait_n(int n) {
  switch (n) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
}

// Shared-memory float2 through volatile accesses, so that a value parked in
// shared memory is not forwarded back into registers by the compiler.  The
// park region is touched by these accesses only, which stay in program order
// (volatile), so they carry no memory clobber: other shared and global
// accesses may be scheduled across them.
__device__ __forceinline__ void st_shared_f2(void* p, float2 v) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ float2 ld_shared_f2(const void* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}

// Streaming 16-byte stores of two rows under one predicate (no branch): the
// rows at a and b, or nothing for a lane whose block lies past the image.
__device__ __forceinline__ void st_pair_cs(void* a, uint4 va, void* b, uint4 vb, bool p) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %10, 0;\n\t"
      "@q st.global.cs.v4.u32 [%0], {%2, %3, %4, %5};\n\t"
      "@q st.global.cs.v4.u32 [%1], {%6, %7, %8, %9};\n\t}" ::"l"(a),
      "l"(b), "r"(va.x), "r"(va.y), "r"(va.z), "r"(va.w), "r"(vb.x), "r"(vb.y), "r"(vb.z), "r"(vb.w), "r"(int(p))
      : "memory");
}

// As st_pair_cs with a predicate per row.
__device__ __forceinline__ void st_pair_cs2(void* a, uint4 va, bool pa, void* b, uint4 vb, bool pb) {
  asm volatile(
      "{\n\t.reg .pred q, r;\n\tsetp.ne.b32 q, %10, 0;\n\tsetp.ne.b32 r, %11, 0;\n\t"
      "@q st.global.cs.v4.u32 [%0], {%2, %3, %4, %5};\n\t"
      "@r st.global.cs.v4.u32 [%1], {%6, %7, %8, %9};\n\t}" ::"l"(a),
      "l"(b), "r"(va.x), "r"(va.y), "r"(va.z), "r"(va.w), "r"(vb.x), "r"(vb.y), "r"(vb.z), "r"(vb.w), "r"(int(pa)),
      "r"(int(pb))
      : "memory");
}

// Alternative configurations of each class's work-list kernel, timed against
// the default (variant 0, the settings above) by the plan autotuner: warps
// per CTA, resident CTAs per SM, parked column pairs, input stages.
template <int C, int VAR>
struct BtAlt;
template <>
struct BtAlt<0, 1> {
  static constexpr int kWarps = 4, kMinCtas = 4, kPark = 1, kStages = 1;
};
template <>
struct BtAlt<0, 2> {
  static constexpr int kWarps = 2, kMinCtas = 5, kPark = 1, kStages = 2;
};
template <>
struct BtAlt<1, 1> {
  static constexpr int kWarps = 1, kMinCtas = 16, kPark = 1, kStages = 1;
};
template <>
struct BtAlt<1, 2> {
  static constexpr int kWarps = 1, kMinCtas = 12, kPark = 0, kStages = 1;
};
template <>
struct BtAlt<2, 1> {
  static constexpr int kWarps = 4, kMinCtas = 3, kPark = 2, kStages = 1;
};
template <>
struct BtAlt<2, 2> {
  static constexpr int kWarps = 1, kMinCtas = 12, kPark = 1, kStages = 1;
};
template <>
struct BtAlt<3, 1> {
  static constexpr int kWarps = 1, kMinCtas = 12, kPark = 1, kStages = 1;
};
template <>
struct BtAlt<3, 2> {
  static constexpr int kWarps = 4, kMinCtas = 3, kPark = 2, kStages = 1;
};
template <>
struct BtAlt<4, 1> {
  static constexpr int kWarps = 1, kMinCtas = 8, kPark = 1, kStages = 1;
};
template <>
struct BtAlt<4, 2> {
  static constexpr int kWarps = 2, kMinCtas = 4, kPark = 3, kStages = 1;
};
template <>
struct BtAlt<5, 1> {
  static constexpr int kWarps = 1, kMinCtas = 8, kPark = 2, kStages = 1;
};
template <>
struct BtAlt<5, 2> {
  static constexpr int kWarps = 2, kMinCtas = 4, kPark = 3, kStages = 1;
};
constexpr int kBtVariants = 3;

// Settings of class C, variant VAR, for SB-byte samples.  16-bit samples
// (classes A..C, variant 0 only): TX16_BT16_WARPS warps per CTA,
// TX16_BT16_MINCTAS CTAs, one stage, TX16_BT16_PARK_A parked pairs in class A
// and TX16_BT16_PARK in B and C.  Measured on 3840x2160 10-bit frames at
// r = 16 (Mblocks/s): 4-warp CTAs x 3, none parked, 4389; x 2 with one
// parked 4306; x 3 with one parked 4310; 1-warp CTAs x 8, none parked, 4347;
// class A (r = 4) with none parked 4499 against 4401 with one.
#ifndef TX16_BT16_WARPS
#define TX16_BT16_WARPS 4
#endif
#ifndef TX16_BT16_MINCTAS
#define TX16_BT16_MINCTAS 3
#endif
#ifndef TX16_BT16_PARK
#define TX16_BT16_PARK 0
#endif
#ifndef TX16_BT16_PARK_A
#define TX16_BT16_PARK_A 0
#endif
// Single-stage refill: bit 0 for 8-bit samples, bit 1 for 16-bit samples.
// Set: the next tile's rows are fetched pair by pair during the inverse pass
// ("rolling"); clear: all 16 after the tile.
#ifndef TX16_BT_ROLLING
#define TX16_BT_ROLLING 2
#endif
template <int C, int VAR>
struct BtSel {
  static constexpr int kWarps = BtAlt<C, VAR>::kWarps, kMinCtas = BtAlt<C, VAR>::kMinCtas,
                       kPark = BtAlt<C, VAR>::kPark, kStages = BtAlt<C, VAR>::kStages;
};
template <int C>
struct BtSel<C, 0> {
  static constexpr int kWarps = BtLimits<C>::kWarps, kMinCtas = BtLimits<C>::kMinCtas, kPark = BtLimits<C>::kPark,
                       kStages = TX16_BT_STAGES;
};
template <int C, int VAR, int SB>
struct BtCfg {
  static constexpr int kWarps = SB == 1 ? BtSel<C, VAR>::kWarps : TX16_BT16_WARPS;
  static constexpr int kMinCtas = SB == 1 ? BtSel<C, VAR>::kMinCtas : TX16_BT16_MINCTAS;
  static constexpr int kPark =
      SB == 1 ? BtSel<C, VAR>::kPark
              : (C == 0 ? TX16_BT16_PARK_A : TX16_BT16_PARK);
  static constexpr int kStages = SB == 1 ? BtSel<C, VAR>::kStages : 1;
  static constexpr bool kRolling = kStages == 1 && ((TX16_BT_ROLLING >> (SB - 1)) & 1) != 0;
  // input rows: per thread 16 rows of 16 SB bytes per stage; parked pairs:
  // 16 float2 per thread and pair
  static constexpr int kStageBytes = 16 * 32 * kWarps * 16 * SB;
  static constexpr int kParkBytes = kPark * 16 * 32 * kWarps * 8;
  static constexpr size_t kSmem = size_t(kStages) * size_t(kStageBytes) + size_t(kParkBytes);
};

// f(integral_constant<int, i>) for i = 0 .. N-1 in order (compile-time indices)
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Tile schedules of one warp (every call is warp-uniform).  StaticWarps: warp
// w takes tiles w, w + W, w + 2W, ... (W warps in the grid).  ChunkWarps:
// warp w takes a contiguous run of tiles.  DynamicWarps: the warp claims
// chunks of tiles from a counter of the work list, the next chunk one chunk
// ahead, so that the next tile is known while this one runs.  A batch launch
// takes ChunkWarps (TX16_BT_CHUNKED 1): 10386-10484 against 10180-10188
// Mblocks/s on 1920x1088 frames at r = 16 with StaticWarps, which changes
// image, and so refills the quantiser table, at nearly every tile.
#ifndef TX16_BT_CHUNKED
#define TX16_BT_CHUNKED 1
#endif
struct StaticWarps {
  int t0, step, ntiles;
  __device__ __forceinline__ int first() const { return t0 < ntiles ? t0 : -1; }
  __device__ __forceinline__ int next(int t) const { return t + step < ntiles ? t + step : -1; }
};

// Warp w of W takes the contiguous tiles [w n / W, (w + 1) n / W): a warp
// changes image (and refills its quantiser tables) about once per launch,
// where taking tiles w, w + W, ... changes image at nearly every tile once
// the images have fewer tiles than the grid has warps (7362 against 6480
// Mregions/s on 1920x1088 frames).
struct ChunkWarps {
  int t0, t1;
  __device__ ChunkWarps(int w, int nw, int ntiles)
      : t0(int(int64_t(w) * ntiles / nw)), t1(int(int64_t(w + 1) * ntiles / nw)) {}
  __device__ __forceinline__ int first() const { return t0 < t1 ? t0 : -1; }
  __device__ __forceinline__ int next(int t) const { return t + 1 < t1 ? t + 1 : -1; }
};
// A CTA takes the contiguous tiles [c n / C, (c + 1) n / C) and its warps
// take them in turn (warp j: start + j, start + j + W, ...), so the warps of
// a CTA read adjacent tiles: the batch launch's schedule (TX16_BT_CTA_RUNS
// 1).  Against one run per warp: r = 4 11373 against about 11200 Mblocks/s,
// r = 16 11180 against 11109-11133, r = 32 equal; the same for 1-warp CTAs.
struct CtaChunkWarps {
  int t, end, step;
  __device__ CtaChunkWarps(int cta, int nctas, int warp, int warps, int ntiles)
      : t(int(int64_t(cta) * ntiles / nctas) + warp), end(int(int64_t(cta + 1) * ntiles / nctas)), step(warps) {}
  __device__ __forceinline__ int first() const { return t < end ? t : -1; }
  __device__ __forceinline__ int next(int u) const { return u + step < end ? u + step : -1; }
};
#ifndef TX16_BT_CTA_RUNS
#define TX16_BT_CTA_RUNS 1
#endif

struct DynamicWarps {
  unsigned* counter;
  int ntiles, chunk, cur_end, next_start;
  __device__ __forceinline__ int claim() const {
    unsigned v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(counter, unsigned(chunk));
    return int(__shfl_sync(0xffffffffu, v, 0));
  }
  __device__ __forceinline__ int first() {
    const int s = claim();
    if (s >= ntiles) return -1;
    cur_end = min(s + chunk, ntiles);
    next_start = claim();
    return s;
  }
  __device__ __forceinline__ int next(int t) {
    if (t + 1 < cur_end) return t + 1;
    const int s = next_start;
    if (s >= ntiles) return -1;
    cur_end = min(s + chunk, ntiles);
    next_start = claim();
    return s;
  }
};

// ---------------------------------------------------------------------------
// Bulk-copy staging: the copy engine (cp.async.bulk, completing on an
// mbarrier) fetches a warp's rows, one copy per pixel row of each run of
// consecutive blocks, instead of one 16-byte cp.async per thread and row.
// ---------------------------------------------------------------------------
#ifndef TX16_BT_BULK
#define TX16_BT_BULK 0
#endif

// Set (bit 0) when a wait for staged rows ran out of time: the warp stopped
// and the launch's results are not valid.  Read by bt_device_errors().
__device__ unsigned g_bt_errors = 0u;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the given phase of m to complete; false if it has not after about
// half a second (nothing in this kernel should ever take that long).
__device__ __noinline__ bool mbar_wait(uint64_t* m, unsigned phase) {
  if (mbar_try_wait(m, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(m, phase)) return true;
    if (global_ns() - t0 > 500000000ull) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The 4 * SB words of a staged row at p (its halves `half` bytes apart).
template <int SB>
__device__ __forceinline__ void load_row_at(const uint8_t* p, int half, unsigned (&w)[4 * SB]) {
#pragma unroll
  for (int h = 0; h < SB; ++h) {
    const uint4 v = *reinterpret_cast<const uint4*>(p + h * half);
    w[4 * h] = v.x;
    w[4 * h + 1] = v.y;
    w[4 * h + 2] = v.z;
    w[4 * h + 3] = v.w;
  }
}

// ---------------------------------------------------------------------------
// Row-pair flow.  The row pass takes rows i and 15 - i in the two lanes of a
// float2, so the first butterfly of the column pass (M1: rows i and 15 - i)
// is a scalar addition across the lanes that writes column-pair floats
// directly, and the last butterfly of the inverse column pass writes the
// (row i, row 15 - i) pairs the inverse row pass reads: no register moves
// between the passes.  Samples enter as 2^23 + 256 x, so M1 needs no bias
// correction: every node of the forward transform is then a multiple of 256
// below 2^32 in magnitude (exact in binary32), the column-pass outputs are
// 256 (T X T^t) plus 2^31 at (0, 0), and the 1/256 is folded into the
// quantiser's scale (an exact power of two).
// ---------------------------------------------------------------------------
// 2^23 + 256 x for sample j of a staged row (exact for samples below 2^15)
template <int SB>
__device__ __forceinline__ float sample256(const unsigned (&w)[4 * SB], int j) {
  if (SB == 1) return __uint_as_float(__byte_perm(w[j >> 2], 0x4B000000u, 0x7404u | (unsigned(j & 3) << 4)));
  return __uint_as_float(__byte_perm(w[j >> 1], 0x4B000000u, (j & 1) ? 0x7324u : 0x7104u));
}

// Quantiser constants of the row-pair flow: the column pass's output sign
// and the 1/256 of the sample encoding folded into the scale.
template <int U, int NP>
__device__ __forceinline__ void fill_consts_t(const ImgParam& I, PairConsts<U, NP>& Q, int lane) {
  using FC = FwdColM16;  // output signs (the same in every pruned form)
  const bool quant = (I.flags & kQuantFlag) != 0;
  float* q = reinterpret_cast<float*>(&Q);
  for (int idx = lane; idx < U * 2 * NP; idx += 32) {
    const int u = idx / (2 * NP);
    const int v = idx - u * 2 * NP;  // = 2 c + half
    const int k = scale_class(u) + scale_class(v);
    const float su = FC::sign(u) < 0 ? -1.f : 1.f;
    const float val = quant ? su * (I.f[k] * (1.f / 256.f)) : su * float(1 << k) * (1.f / 65536.f);
    q[idx] = u < int(I.colh[v]) ? val : 0.f;
  }
  constexpr int kPer = 6 * NP;  // floats per g table
  for (int idx = lane; idx < 2 * kPer; idx += 32) {
    const int tab = idx / kPer;
    const int rem = idx - tab * kPer;
    const int e = rem / (2 * NP);
    const int v = rem - e * 2 * NP;
    const int k = e + scale_class(v);
    q[U * 2 * NP + idx] = quant ? (tab == 0 ? I.g[k] : -8388608.f * I.g[k]) : 0.f;
  }
  __syncwarp();
}

// RAGGED: images whose height is not a multiple of 16 (tx16_codec_any_size):
// the descriptor covers the padded block rows, flags bits from
// kBtMissingShift hold the rows missing from the last block row; rows below
// the image read the last row (edge replication), and only the image's rows
// are stored and counted.

template <int C, int VAR, bool DST, int SB, bool RAGGED, class Sched>
__device__ __forceinline__ void bt_tiles_t(const ImgParam* __restrict__ imgs, int nimg, int ntiles,
                                           unsigned long long* sse, Sched& sched) {
  static_assert(SB == 1 || SB == 2, "8- or 16-bit samples");
  using K = BtClass<C>;
  using N = RowNets<K::V>;
  using Cfg = BtCfg<C, VAR, SB>;
  constexpr int kBtWarps = Cfg::kWarps;
  constexpr int kBtThreads = 32 * kBtWarps;
  constexpr int kStageBytes = Cfg::kStageBytes;
  constexpr int kSlot = kBtThreads * 16;         // bytes of one staged slot
  constexpr int kPark = Cfg::kPark;              // column pairs parked in shared memory
  constexpr int kParkStride = kBtThreads * 8;    // bytes of one parked float2 slot
  constexpr int V = K::V;
  constexpr int U = K::U;
  constexpr int NP = V / 2;
  static_assert(kPark < NP, "at least one column pair stays in registers");
  extern __shared__ __align__(16) uint8_t rows_smem[];
  __shared__ PairConsts<U, NP> consts[kBtWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  PairConsts<U, NP>& Q = consts[wib];
  int t = sched.first();
  if (t < 0) return;
  constexpr int kStages = Cfg::kStages;
  static_assert(kStages == 1 || kStages == 2, "one or two input stages");
  // bulk staging: per warp [row][lane][16 SB bytes] (a row of 32 blocks is
  // contiguous, one copy per run of blocks); cp.async staging: per CTA
  // [row][half][thread][16 bytes]
  constexpr bool kBulk = TX16_BT_BULK != 0;
  constexpr bool kRolling = !kBulk && Cfg::kRolling;
  static_assert(!(kBulk && RAGGED), "the bulk-copy staging reads whole blocks: no ragged images");
  constexpr int kWarpStage = 16 * 32 * 16 * SB;  // bytes of one warp's stage (bulk layout)
  constexpr int kRowStride = kBulk ? 32 * 16 * SB : SB * kSlot;
  constexpr int kHalfStride = kBulk ? 16 : kSlot;
  uint8_t* const park = rows_smem + kStages * kStageBytes + threadIdx.x * 8;
  __shared__ uint64_t mbar[kBulk ? kStages * kBtWarps : 1];
  unsigned phase_bits = 0;  // bit st: parity of the next completion of stage st (bulk staging)
  if (kBulk) {
    if (lane < kStages) mbar_init(&mbar[lane * kBtWarps + wib], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
  }
  auto stage_rows = [&](int st) -> uint8_t* {  // this thread's row 0 of stage st
    return kBulk ? rows_smem + st * kStageBytes + wib * kWarpStage + lane * 16 * SB
                 : rows_smem + st * kStageBytes + threadIdx.x * 16;
  };
  // bulk copies of the rows of this warp's tile tt (image kk) into stage st:
  // lane l copies pixel row l & 15 of the runs l >> 4, (l >> 4) + 2, ... (a
  // run: the tile's blocks in one block row; two runs at most when the image
  // is at least 32 blocks wide)
  auto issue_bulk = [&](int kk, int tt, int st) {
    const ImgParam& I = imgs[kk];
    const int b0 = (tt - I.tile0) * kWarpTile;
    const int nvalid = min(kWarpTile, I.nblk - b0);
    const int2 f = block_coords(I.div_magic, I.nbx, b0);
    const int2 e = block_coords(I.div_magic, I.nbx, b0 + nvalid - 1);
    const int nrun = e.x - f.x + 1;
    const int first = min(nvalid, I.nbx - f.y);  // blocks in the first run
    uint64_t* mb = &mbar[st * kBtWarps + wib];
    uint8_t* wst = rows_smem + st * kStageBytes + wib * kWarpStage;
    __syncwarp();
    fence_proxy_async_smem();  // the stage's earlier reads come before the copies' writes
    if (lane == 0) mbar_expect_tx(mb, unsigned(nvalid) * 256u * SB);
    const int row = lane & 15;
    const uint8_t* src = static_cast<const uint8_t*>(I.src);
    for (int s = lane >> 4; s < nrun; s += 2) {
      const int l0 = s == 0 ? 0 : first + (s - 1) * I.nbx;
      const int len = min(nvalid, s == 0 ? first : l0 + I.nbx) - l0;
      const int col = s == 0 ? f.y : 0;
      bulk_g2s(wst + row * kRowStride + l0 * 16 * SB,
               src + (int64_t(f.x + s) * 16 + row) * I.src_pitch + int64_t(col) * 16 * SB, unsigned(len) * 16u * SB,
               mb);
    }
  };
  // waits for stage st; false if the wait ran out (error recorded)
  auto wait_bulk = [&](int st) -> bool {
    const bool ok = mbar_wait(&mbar[st * kBtWarps + wib], (phase_bits >> st) & 1u);
    phase_bits ^= 1u << st;
    if (!ok && lane == 0) atomicOr(&g_bt_errors, 1u);
    return ok;
  };

  struct RowSrc {
    const uint8_t* g;
    int64_t pitch;
    int bytes;
    int last;  // last row of the block inside the image (RAGGED), else 15
  };
  // last row of block blk of image I inside the image
  auto last_row = [&](const ImgParam& I, int blk) {
    return (RAGGED && blk >= I.nblk - I.nbx) ? 15 - ((I.flags >> kBtMissingShift) & 15) : 15;
  };
  auto row_src = [&](int kk, int tt) {
    const ImgParam& I = imgs[kk];
    const int blk = (tt - I.tile0) * kWarpTile + lane;
    const uint8_t* src = static_cast<const uint8_t*>(I.src);
    if (blk >= I.nblk) return RowSrc{src, 0, 0, 15};
    const int2 c = block_coords(I.div_magic, I.nbx, blk);
    return RowSrc{src + int64_t(c.x) * 16 * I.src_pitch + c.y * 16 * SB, I.src_pitch, 16, last_row(I, blk)};
  };
  auto fetch_row = [&](const RowSrc& r, uint8_t* s, int i) {
    const int64_t row = RAGGED ? min(i, r.last) : i;  // rows below the image repeat its last row
#pragma unroll
    for (int h = 0; h < SB; ++h) cp_async16(s + (i * SB + h) * kSlot, r.g + row * r.pitch + 16 * h, r.bytes);
  };
  // all 16 rows of this thread's block of tile tt (image kk) into stage st, one group
  auto prefetch = [&](int kk, int tt, int st) {
    if (kBulk) {
      issue_bulk(kk, tt, st);
      return;
    }
    const RowSrc r = row_src(kk, tt);
    uint8_t* s = rows_smem + st * kStageBytes + threadIdx.x * 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) fetch_row(r, s, i);
    cp_async_commit();
  };
  auto tile_end_of = [&](int kk) { return kk + 1 < nimg ? imgs[kk + 1].tile0 : ntiles; };

  int k = image_of_tile(imgs, nimg, t);
  int kn = k;
  int end_k = tile_end_of(k), end_kn = end_k;
  prefetch(k, t, 0);
  fill_consts_t<U, NP>(imgs[k], Q, lane);
  unsigned long long acc = 0;
  int stage = 0;
  // One stage, rolling refill: the rows (i, 15 - i) of the next tile are
  // fetched as one commit group each as the inverse pass finishes with them,
  // in the order the forward pass of the next tile reads them.
  bool rolling = false;

  while (t >= 0) {
    const int tn = sched.next(t);
    if (tn >= 0 && tn >= end_kn) {
      kn = image_of_tile(imgs, nimg, tn);
      end_kn = tile_end_of(kn);
    }
    if (kBulk) {
      if (kStages == 2 && tn >= 0) prefetch(kn, tn, stage ^ 1);
      if (!wait_bulk(stage)) {
        // the copies did not arrive in time: wait once more (bounded) for
        // those in flight into this warp's stages, then stop
        if (kStages == 2 && tn >= 0) wait_bulk(stage ^ 1);
        return;
      }
    } else if (kStages == 2 && tn >= 0) {
      prefetch(kn, tn, stage ^ 1);
      cp_async_wait<1>();
    } else if (kStages == 2 || !rolling) {
      cp_async_wait<0>();
    }
    const RowSrc next = (kRolling && tn >= 0) ? row_src(kn, tn) : RowSrc{nullptr, 0, 0};
    if (t >= end_k) {  // warp-uniform: a later image
      if (sse) flush_sse(sse, imgs[k].out_index, acc);
      acc = 0;
      k = image_of_tile(imgs, nimg, t);
      end_k = tile_end_of(k);
      __syncwarp();
      fill_consts_t<U, NP>(imgs[k], Q, lane);
    }
    const ImgParam& I = imgs[k];
    const bool quant = (I.flags & kQuantFlag) != 0;
    const int blk = (t - I.tile0) * kWarpTile + lane;
    const bool valid = blk < I.nblk;
    const int2 c = valid ? block_coords(I.div_magic, I.nbx, blk) : make_int2(0, 0);
    const int last = last_row(I, blk);  // 15 unless RAGGED and in the last block row
    const uint8_t* rows = stage_rows(stage);  // row 0 of this thread's block
    const int64_t dpitch = DST ? I.dst_pitch : 0;
    uint8_t* const dblk = DST ? static_cast<uint8_t*>(I.dst) + int64_t(c.x) * 16 * dpitch + c.y * 16 * SB : nullptr;

    // ---- forward row pass on rows (i, 15 - i), then the column M1 across them:
    // A[s][cp] = (a_s at column 2 cp, a_s at column 2 cp + 1), a = M1 (rows)
    float2 A[16][NP];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (kRolling && rolling) cp_async_wait_n(7 - i);  // rows i and 15 - i of this tile have arrived
      unsigned wa[4 * SB], wb[4 * SB];
      load_row_at<SB>(rows + i * kRowStride, kHalfStride, wa);
      load_row_at<SB>(rows + (15 - i) * kRowStride, kHalfStride, wb);
      float2 X[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) X[j] = make_float2(sample256<SB>(wa, j), sample256<SB>(wb, j));
      float2 S[NP], D[NP];
      N::FR::run(X, S, D);
#pragma unroll
      for (int cp = 0; cp < NP; ++cp) {
        if (cp < kPark) {
          st_shared_f2(park + (cp * 16 + i) * kParkStride, S[cp]);
          st_shared_f2(park + (cp * 16 + 15 - i) * kParkStride, D[cp]);
        } else {
          A[i][cp] = S[cp];
          A[15 - i][cp] = D[cp];
        }
      }
    }

    // ---- column pass per column pair (kept rows u < H[cp], the taller of its
    // two columns): forward network after M1, quantiser, inverse network whose
    // last butterfly writes row pairs ----
    float2 Zr[8][V];  // Zr[i][v] = (z_i, z_(15-i)) at column v (pairs kept in registers)
    static_for<NP>([&](auto cpc) {
      constexpr int cp = decltype(cpc)::value;
      constexpr int HC = K::H[cp];
      using CN = ColNets<HC>;
      float2 a[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) a[s] = cp < kPark ? ld_shared_f2(park + (cp * 16 + s) * kParkStride) : A[s][cp];
      float2 n[HC];
      CN::FC::run(a, n);  // n[u] = FC::sign(u) * 256 Y[u][2 cp + lane], plus 2^31 at (0, 0)
      if (cp == 0) n[0].x = __fadd_rn(n[0].x, CN::FC::sign(0) < 0 ? 2147483648.f : -2147483648.f);
      float2 w[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) w[u] = make_float2(0.f, 0.f);
      if (quant) {
#pragma unroll
        for (int u = 0; u < HC; ++u) {
          const int e = scale_class(u);
          const float2 tq = __fmul2_rn(n[u], Q.fs[u][cp]);  // fl32(Y f), true sign
          const float2 aq = make_float2(fabsf(tq.x), fabsf(tq.y));
          const float2 m = __fadd2_rd(__fadd2_rd(aq, f2(0.5f)), f2(8388608.f));  // 2^23 + floor(|t| + 1/2)
          float2 q = __ffma2_rn(m, Q.gg[e][cp], Q.gc[e][cp]);                  // fl32(level * g)
          q.x = __uint_as_float(__float_as_uint(q.x) | (__float_as_uint(tq.x) & 0x80000000u));
          q.y = __uint_as_float(__float_as_uint(q.y) | (__float_as_uint(tq.y) & 0x80000000u));
          w[u] = q;
        }
      } else {
#pragma unroll
        for (int u = 0; u < HC; ++u) w[u] = __fmul2_rn(n[u], Q.fs[u][cp]);
      }
      float2 Zc[8][2];
      CN::IC::run(w, Zc);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (cp < kPark) st_shared_f2(park + (cp * 16 + 2 * i + h) * kParkStride, Zc[i][h]);
          else Zr[i][2 * cp + h] = Zc[i][h];
        }
    });

    // ---- inverse row pass on rows (i, 15 - i), rounding, stores, SSE ----
    unsigned s1 = 0;  // squared error of this tile's block
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float2 wv[16];
#pragma unroll
      for (int v = 0; v < 16; ++v) {
        if (v < V) {
          const int cp = v >> 1;
          wv[v] = cp < kPark ? ld_shared_f2(park + (cp * 16 + 2 * i + (v & 1)) * kParkStride) : Zr[i][v];
        } else {
          wv[v] = make_float2(0.f, 0.f);
        }
      }
      float2 z[16];
      N::IR::run(wv, z);  // z[j] = sign[j] * (X_tilde[i][j], X_tilde[15 - i][j])
      if (SB == 1) {
        int na[16], nb[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 r = N::IR::sign(j) >= 0 ? __fadd2_rd(z[j], f2(0.5f)) : sub2_rd(f2(0.5f), z[j]);
          const float2 nn = floor_bits2(r);
          na[j] = __float_as_int(nn.x);
          nb[j] = __float_as_int(nn.y);
        }
        unsigned xa[4], xb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xa[q] = pack4_sat_u8(na[4 * q], na[4 * q + 1], na[4 * q + 2], na[4 * q + 3]);
          xb[q] = pack4_sat_u8(nb[4 * q], nb[4 * q + 1], nb[4 * q + 2], nb[4 * q + 3]);
        }
        if (DST && !RAGGED)
          st_pair_cs(dblk + i * dpitch, make_uint4(xa[0], xa[1], xa[2], xa[3]), dblk + (15 - i) * dpitch,
                     make_uint4(xb[0], xb[1], xb[2], xb[3]), valid);
        if (DST && RAGGED)
          st_pair_cs2(dblk + i * dpitch, make_uint4(xa[0], xa[1], xa[2], xa[3]), valid && i <= last,
                      dblk + (15 - i) * dpitch, make_uint4(xb[0], xb[1], xb[2], xb[3]), valid && 15 - i <= last);
        // SSE = sum |x - y|^2 by bytes (vabsdiff4, then dp4a); the error of a
        // block past the image's end is dropped below, and of rows below the
        // image here
        const uint4 ra = *reinterpret_cast<const uint4*>(rows + i * kRowStride);
        const uint4 rb = *reinterpret_cast<const uint4*>(rows + (15 - i) * kRowStride);
        const unsigned ia[4] = {ra.x, ra.y, ra.z, ra.w}, ib[4] = {rb.x, rb.y, rb.z, rb.w};
        unsigned sa = 0, sb = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const unsigned da = __vabsdiffu4(ia[q], xa[q]), db = __vabsdiffu4(ib[q], xb[q]);
          sa = __dp4a(da, da, sa);
          sb = __dp4a(db, db, sb);
        }
        s1 += (!RAGGED || i <= last) ? sa : 0u;
        s1 += (!RAGGED || 15 - i <= last) ? sb : 0u;
      } else {
        const unsigned peak2 = ((1u << (imgs[k].flags & 0xff)) - 1u) * 0x10001u;
        unsigned ya[8], yb[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          int va[2], vb[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float2 r = N::IR::sign(j + e) >= 0 ? __fadd2_rd(z[j + e], f2(0.5f)) : sub2_rd(f2(0.5f), z[j + e]);
            const float2 nn = floor_bits2(r);
            va[e] = __float_as_int(nn.x);
            vb[e] = __float_as_int(nn.y);
          }
          ya[j >> 1] = pack2_sat_u16(va[0], va[1], peak2);
          yb[j >> 1] = pack2_sat_u16(vb[0], vb[1], peak2);
        }
        if (DST) {
          uint8_t* da_ = dblk + i * dpitch;
          uint8_t* db_ = dblk + (15 - i) * dpitch;
          const bool pa = valid && (!RAGGED || i <= last), pb = valid && (!RAGGED || 15 - i <= last);
          st_pair_cs(da_, make_uint4(ya[0], ya[1], ya[2], ya[3]), da_ + 16, make_uint4(ya[4], ya[5], ya[6], ya[7]),
                     pa);
          st_pair_cs(db_, make_uint4(yb[0], yb[1], yb[2], yb[3]), db_ + 16, make_uint4(yb[4], yb[5], yb[6], yb[7]),
                     pb);
        }
        unsigned wa[8], wb[8];
        load_row_at<2>(rows + i * kRowStride, kHalfStride, wa);
        load_row_at<2>(rows + (15 - i) * kRowStride, kHalfStride, wb);
        unsigned sa = 0, sb = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int d0 = int(wa[q] & 0xffffu) - int(ya[q] & 0xffffu), d1 = int(wa[q] >> 16) - int(ya[q] >> 16);
          const int d2 = int(wb[q] & 0xffffu) - int(yb[q] & 0xffffu), d3 = int(wb[q] >> 16) - int(yb[q] >> 16);
          sa += unsigned(d0 * d0) + unsigned(d1 * d1);
          sb += unsigned(d2 * d2) + unsigned(d3 * d3);
        }
        s1 += (!RAGGED || i <= last) ? sa : 0u;
        s1 += (!RAGGED || 15 - i <= last) ? sb : 0u;
      }
      // rows i and 15 - i of the stage are used: refill them for the next tile
      if (kRolling && tn >= 0) {
        uint8_t* s = rows_smem + threadIdx.x * 16;
        fetch_row(next, s, i);
        fetch_row(next, s, 15 - i);
        cp_async_commit();
      }
    }
    // bulk staging leaves the rows of blocks past the image's end as they
    // were: those lanes' squared error is dropped
    acc += (kBulk && !valid) ? 0u : s1;
    if (kStages == 1 && !kRolling && tn >= 0) prefetch(kn, tn, 0);
    rolling = kRolling && tn >= 0;
    t = tn;
    stage ^= (kStages - 1);
  }
  if (sse) flush_sse(sse, imgs[k].out_index, acc);
}

template <int MAXI, int C, bool DST, int SB, bool RAGGED = false>
__global__ void __launch_bounds__(32 * BtCfg<C, 0, SB>::kWarps, BtCfg<C, 0, SB>::kMinCtas)
    fused_bt_kernel(const __grid_constant__ BatchParams<MAXI> P) {
  const int w = int(blockIdx.x) * BtCfg<C, 0, SB>::kWarps + int(threadIdx.x >> 5);
  const int nw = int(gridDim.x) * BtCfg<C, 0, SB>::kWarps;
  if (TX16_BT_CTA_RUNS) {
    CtaChunkWarps sched(int(blockIdx.x), int(gridDim.x), int(threadIdx.x >> 5), BtCfg<C, 0, SB>::kWarps, P.ntiles);
    bt_tiles_t<C, 0, DST, SB, RAGGED>(P.img, P.nimg, P.ntiles, P.sse, sched);
  } else if (TX16_BT_CHUNKED) {
    ChunkWarps sched(w, nw, P.ntiles);
    bt_tiles_t<C, 0, DST, SB, RAGGED>(P.img, P.nimg, P.ntiles, P.sse, sched);
  } else {
    StaticWarps sched{w, nw, P.ntiles};
    bt_tiles_t<C, 0, DST, SB, RAGGED>(P.img, P.nimg, P.ntiles, P.sse, sched);
  }
}

template <int C, int VAR, bool DST>
__global__ void __launch_bounds__(32 * BtCfg<C, VAR, 1>::kWarps, BtCfg<C, VAR, 1>::kMinCtas)
    fused_bt_list_kernel(const ImgParam* __restrict__ imgs, int nimg, int ntiles, unsigned* counter, int chunk,
                         unsigned long long* sse) {
  if (chunk == 0) {  // static: a contiguous run of tiles per CTA, no claims
    CtaChunkWarps sched(int(blockIdx.x), int(gridDim.x), int(threadIdx.x >> 5), BtCfg<C, VAR, 1>::kWarps, ntiles);
    bt_tiles_t<C, VAR, DST, 1, false>(imgs, nimg, ntiles, sse, sched);
    return;
  }
  DynamicWarps sched{counter, ntiles, chunk, 0, 0};
  bt_tiles_t<C, VAR, DST, 1, false>(imgs, nimg, ntiles, sse, sched);
}

// keep_index: the descriptors' out_index are already the SSE slots (RAGGED
// launches over a subset of a call's images); otherwise image i of the launch
// adds into sse[i].
template <int MAXI, int C, bool DST, int SB, bool RAGGED = false>
tx16_status launch_bt(const ImgParam* imgs, int n, unsigned long long* sse, cudaStream_t stream,
                      bool keep_index = false) {
  using Cfg = BtCfg<C, 0, SB>;
  BatchParams<MAXI> P;
  P.nimg = n;
  P.sse = sse;
  P.coeffs = nullptr;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].tile0 = tiles;
    if (!keep_index) P.img[i].out_index = i;
    tiles += (imgs[i].nblk + kWarpTile - 1) / kWarpTile;
  }
  P.ntiles = tiles;
  constexpr int kBtThreads = 32 * Cfg::kWarps;
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    if (cudaFuncSetAttribute(fused_bt_kernel<MAXI, C, DST, SB, RAGGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(Cfg::kSmem)) != cudaSuccess)
      return TX16_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fused_bt_kernel<MAXI, C, DST, SB, RAGGED>, kBtThreads,
                                                      Cfg::kSmem) != cudaSuccess ||
        o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min((tiles + Cfg::kWarps - 1) / Cfg::kWarps, occ * device_sm_count()));
  fused_bt_kernel<MAXI, C, DST, SB, RAGGED><<<grid, kBtThreads, Cfg::kSmem, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

template <int MAXI, int C, int SB>
tx16_status launch_bt_dst(bool dst, const ImgParam* imgs, int n, unsigned long long* sse, cudaStream_t stream) {
  return dst ? launch_bt<MAXI, C, true, SB>(imgs, n, sse, stream) : launch_bt<MAXI, C, false, SB>(imgs, n, sse, stream);
}

template <int C, int VAR, bool DST>
int bt_list_max_ctas() {
  using Cfg = BtCfg<C, VAR, 1>;
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    auto k = fused_bt_list_kernel<C, VAR, DST>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::kSmem)) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, 32 * Cfg::kWarps, Cfg::kSmem) != cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}

template <int C, int VAR, bool DST>
tx16_status launch_bt_list(const ImgParam* d_imgs, int nimg, int ntiles, unsigned* counter, int chunk,
                           int ctas_per_sm, unsigned long long* sse, cudaStream_t stream) {
  using Cfg = BtCfg<C, VAR, 1>;
  const int occ = bt_list_max_ctas<C, VAR, DST>();
  if (occ == 0) return TX16_ECUDA;
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  const int grid = std::max(1, std::min((ntiles + Cfg::kWarps - 1) / Cfg::kWarps, per_sm * device_sm_count()));
  fused_bt_list_kernel<C, VAR, DST><<<grid, 32 * Cfg::kWarps, Cfg::kSmem, stream>>>(d_imgs, nimg, ntiles, counter,
                                                                                    chunk, sse);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

template <int C, int VAR>
tx16_status launch_bt_list_dst(bool dst, const ImgParam* d_imgs, int nimg, int ntiles, unsigned* counter, int chunk,
                               int ctas_per_sm, unsigned long long* sse, cudaStream_t stream) {
  return dst ? launch_bt_list<C, VAR, true>(d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream)
             : launch_bt_list<C, VAR, false>(d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
}

}  // namespace

// Entry points of one class (explicitly instantiated, one translation unit per
// class: tx16_bt_c<class>.cu).
// A batch whose descriptors travel in the kernel parameters (variant 0); SB =
// 2 (9..12-bit samples) for classes A..C only.
template <int C>
tx16_status bt_batch(bool dst, int sb, const ImgParam* imgs, int n, unsigned long long* sse, cudaStream_t stream) {
  if (sb == 1) {
    if (n <= 8) return launch_bt_dst<8, C, 1>(dst, imgs, n, sse, stream);
    return launch_bt_dst<kMaxImg, C, 1>(dst, imgs, n, sse, stream);
  }
  if constexpr (C <= 2) {
    if (n <= 8) return launch_bt_dst<8, C, 2>(dst, imgs, n, sse, stream);
    return launch_bt_dst<kMaxImg, C, 2>(dst, imgs, n, sse, stream);
  }
  return TX16_EINVAL;
}
// 8-bit images whose out_index are their SSE slots of sse (a subset of a
// call's images, grouped by zonal class), at most kMaxImg.
template <int C>
tx16_status bt_batch_keep(bool dst, const ImgParam* imgs, int n, unsigned long long* sse, cudaStream_t stream) {
  return dst ? launch_bt<kMaxImg, C, true, 1>(imgs, n, sse, stream, true)
             : launch_bt<kMaxImg, C, false, 1>(imgs, n, sse, stream, true);
}
// Images of ragged height (see kBtMissingShift), out_index = SSE slot of sse,
// at most kMaxImg.
template <int C>
tx16_status bt_batch_ragged(bool dst, int sb, const ImgParam* imgs, int n, unsigned long long* sse,
                            cudaStream_t stream) {
  if (sb == 1)
    return dst ? launch_bt<kMaxImg, C, true, 1, true>(imgs, n, sse, stream, true)
               : launch_bt<kMaxImg, C, false, 1, true>(imgs, n, sse, stream, true);
  if constexpr (C <= 2)
    return dst ? launch_bt<kMaxImg, C, true, 2, true>(imgs, n, sse, stream, true)
               : launch_bt<kMaxImg, C, false, 2, true>(imgs, n, sse, stream, true);
  return TX16_EINVAL;
}
// A work list in device memory (tile0 in warp tiles), tiles claimed `chunk` at
// a time, by the kernel of variant `var` (0 .. kBtVariants - 1).
template <int C>
tx16_status bt_list(int var, bool dst, const ImgParam* d_imgs, int nimg, int ntiles, unsigned* counter, int chunk,
                    int ctas_per_sm, unsigned long long* sse, cudaStream_t stream) {
  switch (var) {
    case 0: return launch_bt_list_dst<C, 0>(dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 1: return launch_bt_list_dst<C, 1>(dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 2: return launch_bt_list_dst<C, 2>(dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    default: return TX16_EINVAL;
  }
}
// resident CTAs per SM of variant `var` (0 if it cannot run)
template <int C>
int bt_list_ctas(int var, bool dst) {
  switch (var) {
    case 0: return dst ? bt_list_max_ctas<C, 0, true>() : bt_list_max_ctas<C, 0, false>();
    case 1: return dst ? bt_list_max_ctas<C, 1, true>() : bt_list_max_ctas<C, 1, false>();
    case 2: return dst ? bt_list_max_ctas<C, 2, true>() : bt_list_max_ctas<C, 2, false>();
    default: return 0;
  }
}
// warps per CTA, parked column pairs and input stages of variant `var`
template <int C>
void bt_variant_info(int var, int* warps, int* park, int* stages) {
  switch (var) {
    case 0: *warps = BtSel<C, 0>::kWarps; *park = BtSel<C, 0>::kPark; *stages = BtSel<C, 0>::kStages; break;
    case 1: *warps = BtSel<C, 1>::kWarps; *park = BtSel<C, 1>::kPark; *stages = BtSel<C, 1>::kStages; break;
    default: *warps = BtSel<C, 2>::kWarps; *park = BtSel<C, 2>::kPark; *stages = BtSel<C, 2>::kStages; break;
  }
}

}  // namespace tx16
