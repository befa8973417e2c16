// Mixed 8/16 tiling, one 16x16 region per thread, entirely in registers: the
// region is coded as one block with T (the one-block-per-thread flow of
// tx16_fused_bt.cuh) and as four 8x8 blocks with T8 (Sec. 2.1), and the
// tiling with the smaller squared error is stored (ties: 16x16), or the one
// the image forces.  8-bit planes with a quantiser.
//
// Row pairs.  Both paths hold rows i and 15 - i of the region in the two
// lanes of a float2 (i = 0..7).  For the 8x8 blocks, lane x walks the upper
// blocks top-down (row i) and lane y the lower blocks bottom-up (row 7 - i of
// the lower block), so the T8 column network runs on the eight row pairs in
// order with no exchange: its first stage (M2's first half) pairs rows k and
// 7 - k of a block, which are row pairs k and 7 - k in either lane; lane y
// then carries the odd frequencies negated, which the odd-symmetric quantiser
// keeps and the inverse column network's last stage undoes, returning the
// (i, 15 - i) pairing with true values.
//
// Per region:
//   8x8 path   per half (columns 0..7, 8..15): T8 row pass on the eight row
//              pairs, T8 column pass per kept column, quantiser, inverse
//              column and row passes, rounding; the reconstruction goes to a
//              second shared-memory buffer and its squared error is summed
//   16x16 path the one-block-per-thread flow; its reconstruction overwrites
//              the staged input rows once their squared error is taken
//   choice     the rows of the chosen reconstruction are stored from shared
//              memory, and the staged rows are refilled with the next tile
//
// Exactness is that of the one-block-per-thread kernel on both paths: samples
// enter as 2^23 + 256 x, every forward node is a multiple of 256 below 2^32
// (the 8x8 DC carries 64 * 2^23 = 2^29, removed exactly), the 1/256 is folded
// into the quantiser's scale, and the inverse networks follow the library's
// binary32 definition stage by stage.
#pragma once

#include "tx16_fused_bt.cuh"

namespace tx16 {
namespace {

// Zonal classes of the 8x8 path: per kept column v of an 8x8 block, its kept
// rows H8[v] (the column heights of the 8x8 zig-zag zone Z_rmax).
//   class   0       1
//   r_max   4       16
//   H8      3 1     5 4 3 2 1 1
template <int C8>
struct Mix8Class;
template <>
struct Mix8Class<0> {
  static constexpr int kRmax = 4, V = 2, U = 3;
  static constexpr int H[2] = {3, 1};
};
template <>
struct Mix8Class<1> {
  static constexpr int kRmax = 16, V = 6, U = 5;
  static constexpr int H[6] = {5, 4, 3, 2, 1, 1};
};

// Per class of the 16x16 path: warps per CTA, resident CTAs per SM the
// registers are budgeted for, column pairs parked in shared memory.  The
// second buffer (the 8x8 reconstruction) doubles the staging memory, so CTAs
// per SM stay at or below 12 and the register limit at 168.  Input stages:
// 1, the next tile's rows are fetched pair by pair as the chosen
// reconstruction is stored (the other warps cover the latency); 2, during
// the whole tile (24 KB per warp, 9 warps per SM).  Measured on 1920x1088
// frames, q = 16, r16 = 16, r8 = 4: one stage at 12 warps 7362 Mregions/s,
// two stages at 9 warps 6886.
#ifndef TX16_MIX_WARPS
#define TX16_MIX_WARPS 1
#endif
#ifndef TX16_MIX_MINCTAS
#define TX16_MIX_MINCTAS 12
#endif
#ifndef TX16_MIX_STAGES
#define TX16_MIX_STAGES 1
#endif
#ifndef TX16_MIX_MERGED
#define TX16_MIX_MERGED 1
#endif
template <int C16>
struct MixCfg {
  static constexpr int kWarps = TX16_MIX_WARPS, kMinCtas = TX16_MIX_MINCTAS, kStages = TX16_MIX_STAGES;
  static constexpr int kPark = C16 <= 1 ? 0 : C16 - 1;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kStageBytes = 16 * kThreads * 16;  // 16 rows of 16 bytes per thread
  static constexpr int kParkBytes = kPark * 16 * kThreads * 8;
  // input stages, the 8x8 reconstruction, parked column pairs
  static constexpr size_t kSmem = size_t(kStages + 1) * size_t(kStageBytes) + size_t(kParkBytes);
};

// Quantiser constants of the 8x8 path, the same in both lanes.
template <int U8, int V8>
struct Mix8Consts {
  float2 fs[U8][V8];  // sign f8 / 256; 0 outside the zone
  float2 gg[U8][V8];  // g8
  float2 gc[U8][V8];  // -2^23 g8
};

__device__ __forceinline__ int scale_class8(int u) { return (u & 1) ? 2 : ((u & 2) ? 1 : 0); }  // 0,2,1,2,0,2,1,2

// col_net: the column pass runs the generated T8 network (its output signs
// enter the scale); otherwise it accumulates T8 term by term (true signs).
template <int U8, int V8>
__device__ __forceinline__ void fill_consts8(const MixedParam& M, Mix8Consts<U8, V8>& Q, int lane, bool col_net) {
  for (int idx = lane; idx < U8 * V8; idx += 32) {
    const int u = idx / V8;
    const int v = idx - u * V8;
    const int k = scale_class8(u) + scale_class8(v);
    const float s = FwdRow8T8::sign(v) * (col_net ? FwdCol8M8::sign(u) : 1) < 0 ? -1.f : 1.f;
    const float fs = u < int(M.colh8[v]) ? s * (M.f8[k] * (1.f / 256.f)) : 0.f;
    Q.fs[u][v] = f2(fs);
    Q.gg[u][v] = f2(M.g8[k]);
    Q.gc[u][v] = f2(-8388608.f * M.g8[k]);
  }
  __syncwarp();
}

// 2^23 + 256 x for byte j (0..3) of w
__device__ __forceinline__ float byte256(unsigned w, int j) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7404u | (unsigned(j) << 4)));
}

// Rounded, clamped samples of a pair of lanes, packed: 8 samples per lane
// from z[0..7] with output signs SIGN(j).
template <class IR>
__device__ __forceinline__ void round_pack8(const float2 (&z)[8], unsigned (&a)[2], unsigned (&b)[2]) {
  int na[8], nb[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2 r = IR::sign(j) >= 0 ? __fadd2_rd(z[j], f2(0.5f)) : sub2_rd(f2(0.5f), z[j]);
    const float2 nn = floor_bits2(r);
    na[j] = __float_as_int(nn.x);
    nb[j] = __float_as_int(nn.y);
  }
  a[0] = pack4_sat_u8(na[0], na[1], na[2], na[3]);
  a[1] = pack4_sat_u8(na[4], na[5], na[6], na[7]);
  b[0] = pack4_sat_u8(nb[0], nb[1], nb[2], nb[3]);
  b[1] = pack4_sat_u8(nb[4], nb[5], nb[6], nb[7]);
}

// level -> fl32(level g) with the sign of t (the S-merged quantiser of the
// one-block-per-thread kernel): t = fl32(Y f) with |t| + 1/2 < 2^23
__device__ __forceinline__ float2 quantise_pair(float2 n, float2 fs, float2 gg, float2 gc) {
  const float2 tq = __fmul2_rn(n, fs);
  const float2 aq = make_float2(fabsf(tq.x), fabsf(tq.y));
  const float2 m = __fadd2_rd(__fadd2_rd(aq, f2(0.5f)), f2(8388608.f));  // 2^23 + floor(|t| + 1/2)
  float2 q = __ffma2_rn(m, gg, gc);                                     // fl32(level * g)
  q.x = __uint_as_float(__float_as_uint(q.x) | (__float_as_uint(tq.x) & 0x80000000u));
  q.y = __uint_as_float(__float_as_uint(q.y) | (__float_as_uint(tq.y) & 0x80000000u));
  return q;
}

template <int MAXI>
struct MixedBtBatch {
  int32_t nimg, ntiles;
  unsigned long long* sse;  // indexed by out_index
  uint8_t* split;           // indexed by blk0 + region, or nullptr
  MixedParam img[MAXI];
};
static_assert(sizeof(MixedBtBatch<kMixMaxImg>) < 32000, "kernel parameters too large");

template <int C16, int C8, class Sched>
__device__ __forceinline__ void mixed_tiles(const MixedParam* __restrict__ imgs, int nimg, int ntiles,
                                            unsigned long long* sse, uint8_t* split_map, Sched& sched) {
  using K = BtClass<C16>;
  using N = RowNets<K::V>;
  using K8 = Mix8Class<C8>;
  using N8 = Row8Nets<K8::V>;
  using Cfg = MixCfg<C16>;
  constexpr int kWarps = Cfg::kWarps;
  constexpr int kThreads = Cfg::kThreads;
  constexpr int kSlot = kThreads * 16;  // bytes of one staged row of all threads
  constexpr int kRowStride = kSlot;
  constexpr int kPark = Cfg::kPark;
  constexpr int kParkStride = kThreads * 8;
  constexpr int V = K::V, U = K::U, NP = V / 2;
  constexpr int V8 = K8::V, U8 = K8::U;
  // class 0 (r8 <= 4: four cells per 8x8 block) shares the row loop with the
  // 16x16 path; class 1 keeps a loop of its own (its 16 accumulators per half
  // would not fit beside the 16x16 path's registers)
  constexpr bool kMerged8 = C8 == 0 && TX16_MIX_MERGED;
  static_assert(kPark < NP, "at least one column pair stays in registers");
  extern __shared__ __align__(16) uint8_t mix_smem[];
  __shared__ PairConsts<U, NP> consts16[kWarps];
  __shared__ Mix8Consts<U8, V8> consts8[kWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  PairConsts<U, NP>& Q = consts16[wib];
  Mix8Consts<U8, V8>& Q8 = consts8[wib];
  constexpr int kStages = Cfg::kStages;
  static_assert(kStages == 1 || kStages == 2, "one or two input stages");
  // per stage: input rows, then the T reconstruction
  uint8_t* const xrows0 = mix_smem + threadIdx.x * 16;
  uint8_t* const rows8 = mix_smem + kStages * Cfg::kStageBytes + threadIdx.x * 16;  // the T8 reconstruction
  uint8_t* const park = mix_smem + (kStages + 1) * Cfg::kStageBytes + threadIdx.x * 8;  // parked column pairs
  int t = sched.first();
  if (t < 0) return;

  struct RowSrc {
    const uint8_t* g;
    int64_t pitch;
    int bytes;
  };
  auto row_src = [&](int kk, int tt) {
    const ImgParam& I = imgs[kk].p;
    const int blk = (tt - I.tile0) * kWarpTile + lane;
    const uint8_t* src = static_cast<const uint8_t*>(I.src);
    if (blk >= I.nblk) return RowSrc{src, 0, 0};
    const int2 c = block_coords(I.div_magic, I.nbx, blk);
    return RowSrc{src + int64_t(c.x) * 16 * I.src_pitch + c.y * 16, I.src_pitch, 16};
  };
  auto fetch_row = [&](const RowSrc& r, uint8_t* xr, int i) {
    cp_async16(xr + i * kRowStride, r.g + i * r.pitch, r.bytes);
  };
  auto image_of = [&](int tt) {  // binary search; tile0 ascending
    int lo = 0, hi = nimg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (imgs[mid].p.tile0 <= tt) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  auto tile_end_of = [&](int kk) { return kk + 1 < nimg ? imgs[kk + 1].p.tile0 : ntiles; };

  int k = image_of(t);
  int kn = k;
  int end_k = tile_end_of(k), end_kn = end_k;
  auto prefetch = [&](int kk, int tt, int st) {  // all 16 rows of tile tt into stage st, one group
    const RowSrc r = row_src(kk, tt);
#pragma unroll
    for (int i = 0; i < 16; ++i) fetch_row(r, xrows0 + st * Cfg::kStageBytes, i);
    cp_async_commit();
  };
  prefetch(k, t, 0);
  int stage = 0;
  fill_consts_t<U, NP>(imgs[k].p, Q, lane);
  fill_consts8<U8, V8>(imgs[k], Q8, lane, !kMerged8);
  unsigned long long acc = 0;
  bool rolling = false;  // the rows arrive pair by pair (one commit group per pair)

  while (t >= 0) {
    const int tn = sched.next(t);
    if (tn >= 0 && tn >= end_kn) {
      kn = image_of(tn);
      end_kn = tile_end_of(kn);
    }
    if (kStages == 2 && tn >= 0) {
      prefetch(kn, tn, stage ^ 1);
      cp_async_wait<1>();
    } else if (kStages == 2 || !rolling) {
      cp_async_wait<0>();
    }
    uint8_t* const xrows = xrows0 + stage * Cfg::kStageBytes;
    const RowSrc next = (kStages == 1 && tn >= 0) ? row_src(kn, tn) : RowSrc{nullptr, 0, 0};
    if (t >= end_k) {  // warp-uniform: a later image
      if (sse) flush_sse(sse, imgs[k].p.out_index, acc);
      acc = 0;
      k = image_of(t);
      end_k = tile_end_of(k);
      __syncwarp();
      fill_consts_t<U, NP>(imgs[k].p, Q, lane);
      fill_consts8<U8, V8>(imgs[k], Q8, lane, !kMerged8);
    }
    const MixedParam& M = imgs[k];
    const ImgParam& I = M.p;
    const int blk = (t - I.tile0) * kWarpTile + lane;
    const bool valid = blk < I.nblk;
    const int2 c = valid ? block_coords(I.div_magic, I.nbx, blk) : make_int2(0, 0);
    uint8_t* const dblk = static_cast<uint8_t*>(I.dst) + int64_t(c.x) * 16 * I.dst_pitch + c.y * 16;

    // ---- the 8x8 path after its column pass, per half hh: n_of(v, n) gives
    // n[u] = sign * 256 Y8[u][v] per lane (u < H8[v]; lane y: odd u negated),
    // the 2^29 of the DC already removed.  Quantiser, inverse column and row
    // passes, rounding, squared error, the reconstruction into rows8.
    auto finish8 = [&](int hh, auto&& n_of) -> unsigned {
      unsigned e = 0;
      float2 Z8[8][V8];  // Z8[m][v] = (row m of the upper block, row 7 - m of the lower) at column v
      static_for<V8>([&](auto vc) {
        constexpr int v = decltype(vc)::value;
        constexpr int H = K8::H[v];
        using CN = Col8Nets<H>;
        float2 n[H];
        n_of(vc, n);
        float2 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < H; ++u) w[u] = quantise_pair(n[u], Q8.fs[u][v], Q8.gg[u][v], Q8.gc[u][v]);
        float2 z[8];
        CN::IC::run(w, z);
#pragma unroll
        for (int m = 0; m < 8; ++m) Z8[m][v] = z[m];
      });
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        float2 wv[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) wv[v] = v < V8 ? Z8[m][v] : make_float2(0.f, 0.f);
        float2 z[8];
        N8::IR::run(wv, z);  // z[j] = sign[j] * (row m, row 15 - m) at column 8 hh + j
        unsigned pa[2], pb[2];
        round_pack8<typename N8::IR>(z, pa, pb);
        const uint2 xa = *reinterpret_cast<const uint2*>(xrows + m * kRowStride + 8 * hh);
        const uint2 xb = *reinterpret_cast<const uint2*>(xrows + (15 - m) * kRowStride + 8 * hh);
        unsigned d = __vabsdiffu4(xa.x, pa[0]);
        e = __dp4a(d, d, e);
        d = __vabsdiffu4(xa.y, pa[1]);
        e = __dp4a(d, d, e);
        d = __vabsdiffu4(xb.x, pb[0]);
        e = __dp4a(d, d, e);
        d = __vabsdiffu4(xb.y, pb[1]);
        e = __dp4a(d, d, e);
        *reinterpret_cast<uint2*>(rows8 + m * kRowStride + 8 * hh) = make_uint2(pa[0], pa[1]);
        *reinterpret_cast<uint2*>(rows8 + (15 - m) * kRowStride + 8 * hh) = make_uint2(pb[0], pb[1]);
      }
      return e;
    };
    // ---- the 16x16 row pass of rows (i, 15 - i) from their unpacked samples
    float2 A[16][NP];
    auto row16 = [&](int i, const float2 (&X)[16]) {
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
    };
    constexpr float kDc8 = FwdRow8T8::sign(0) * (kMerged8 ? 1 : FwdCol8M8::sign(0)) < 0 ? 536870912.f : -536870912.f;
    unsigned e8 = 0;
    if constexpr (kMerged8) {
      // ==== one row loop for both paths: the samples are unpacked once; the
      // 8x8 column pass accumulates T8 down the row pairs term by term (exact:
      // every value is an integer multiple of 256 below 2^32)
      float2 Y8[2][V8][U8];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int v = 0; v < V8; ++v)
#pragma unroll
          for (int u = 0; u < U8; ++u) Y8[hh][v][u] = make_float2(0.f, 0.f);
      static_for<8>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if (kStages == 1 && rolling) cp_async_wait_n(7 - i);  // rows i and 15 - i have arrived
        unsigned wa[4], wb[4];
        load_row_at<1>(xrows + i * kRowStride, kSlot, wa);
        load_row_at<1>(xrows + (15 - i) * kRowStride, kSlot, wb);
        float2 X[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) X[j] = make_float2(sample256<1>(wa, j), sample256<1>(wb, j));
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float2 Rr[V8];
          N8::FR::run(reinterpret_cast<const float2(&)[8]>(X[8 * hh]), Rr);
          static_for<V8>([&](auto vc) {
            constexpr int v = decltype(vc)::value;
            static_for<U8>([&](auto uc) {
              constexpr int u = decltype(uc)::value;
              constexpr int c = u < K8::H[v] ? kT8[u][i] : 0;
              if constexpr (c > 0) Y8[hh][v][u] = __fadd2_rn(Y8[hh][v][u], Rr[v]);
              if constexpr (c < 0) Y8[hh][v][u] = sub2(Y8[hh][v][u], Rr[v]);
            });
          });
        }
        row16(i, X);
      });
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
        e8 += finish8(hh, [&](auto vc, auto& n) {
          constexpr int v = decltype(vc)::value;
          constexpr int Hv = K8::H[v];
#pragma unroll
          for (int u = 0; u < Hv; ++u) n[u] = Y8[hh][v][u];
          if (v == 0) n[0] = __fadd2_rn(n[0], f2(kDc8));
        });
    } else {
      // ==== the 8x8 path on its own, one half at a time: T8 row pass, T8
      // column networks; then the 16x16 row loop
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float2 R[8][V8];  // R[i][v]: T8 row outputs of rows (i, 15 - i), half hh
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (kStages == 1 && hh == 0 && rolling) cp_async_wait_n(7 - i);  // rows i and 15 - i have arrived
          const uint2 wa = *reinterpret_cast<const uint2*>(xrows + i * kRowStride + 8 * hh);
          const uint2 wb = *reinterpret_cast<const uint2*>(xrows + (15 - i) * kRowStride + 8 * hh);
          float2 X[8];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            X[j] = make_float2(byte256(wa.x, j), byte256(wb.x, j));
            X[4 + j] = make_float2(byte256(wa.y, j), byte256(wb.y, j));
          }
          float2 Rr[V8];
          N8::FR::run(X, Rr);
#pragma unroll
          for (int v = 0; v < V8; ++v) R[i][v] = Rr[v];
        }
        e8 += finish8(hh, [&](auto vc, auto& n) {
          constexpr int v = decltype(vc)::value;
          float2 a[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) a[i] = R[i][v];
          constexpr int Hv = K8::H[v];
          Col8Nets<Hv>::FC::run(a, n);  // n[u] = sign * 256 Y8[u][v] per lane, plus 2^29 at (0, 0)
          if (v == 0) n[0] = __fadd2_rn(n[0], f2(kDc8));
        });
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        unsigned wa[4], wb[4];
        load_row_at<1>(xrows + i * kRowStride, kSlot, wa);
        load_row_at<1>(xrows + (15 - i) * kRowStride, kSlot, wb);
        float2 X[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) X[j] = make_float2(sample256<1>(wa, j), sample256<1>(wb, j));
        row16(i, X);
      }
    }

    // ================= one 16x16 block with T: column pass onwards =================
    float2 Zr[8][V];
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
#pragma unroll
      for (int u = 0; u < HC; ++u) {
        const int e = scale_class(u);
        w[u] = quantise_pair(n[u], Q.fs[u][cp], Q.gg[e][cp], Q.gc[e][cp]);
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
    unsigned e16 = 0;
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
      uint4* const ra = reinterpret_cast<uint4*>(xrows + i * kRowStride);
      uint4* const rb = reinterpret_cast<uint4*>(xrows + (15 - i) * kRowStride);
      const uint4 ia = *ra, ib = *rb;
      const unsigned sa[4] = {ia.x, ia.y, ia.z, ia.w}, sb[4] = {ib.x, ib.y, ib.z, ib.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned da = __vabsdiffu4(sa[q], xa[q]), db = __vabsdiffu4(sb[q], xb[q]);
        e16 = __dp4a(da, da, e16);
        e16 = __dp4a(db, db, e16);
      }
      *ra = make_uint4(xa[0], xa[1], xa[2], xa[3]);  // the input rows are used: keep the reconstruction
      *rb = make_uint4(xb[0], xb[1], xb[2], xb[3]);
    }

    // ================= the chosen tiling: stores, refill, error =================
    const bool split = M.mode == 2 || (M.mode == 0 && e8 < e16);
    const uint8_t* const src = split ? rows8 : xrows;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint4 ra = *reinterpret_cast<const uint4*>(src + i * kRowStride);
      const uint4 rb = *reinterpret_cast<const uint4*>(src + (15 - i) * kRowStride);
      st_pair_cs(dblk + i * I.dst_pitch, ra, dblk + (15 - i) * I.dst_pitch, rb, valid);
      if (kStages == 1 && tn >= 0) {  // rows i and 15 - i of the next tile, one commit group
        fetch_row(next, xrows, i);
        fetch_row(next, xrows, 15 - i);
        cp_async_commit();
      }
    }
    if (valid) {
      if (split_map) split_map[I.blk0 + blk] = split ? 1 : 0;
      acc += split ? e8 : e16;
    }
    rolling = kStages == 1 && tn >= 0;
    t = tn;
    stage ^= (kStages - 1);
  }
  if (sse) flush_sse(sse, imgs[k].p.out_index, acc);
}

#ifndef TX16_MIX_CHUNKED
#define TX16_MIX_CHUNKED 1
#endif

template <int MAXI, int C16, int C8>
__global__ void __launch_bounds__(MixCfg<C16>::kThreads, MixCfg<C16>::kMinCtas)
    mixed_bt_kernel(const __grid_constant__ MixedBtBatch<MAXI> P) {
  const int w = int(blockIdx.x) * MixCfg<C16>::kWarps + int(threadIdx.x >> 5);
  const int nw = int(gridDim.x) * MixCfg<C16>::kWarps;
  if (TX16_MIX_CHUNKED) {
    ChunkWarps sched(w, nw, P.ntiles);
    mixed_tiles<C16, C8>(P.img, P.nimg, P.ntiles, P.sse, P.split, sched);
  } else {
    StaticWarps sched{w, nw, P.ntiles};
    mixed_tiles<C16, C8>(P.img, P.nimg, P.ntiles, P.sse, P.split, sched);
  }
}

}  // namespace

// One launch over images of one class pair (at most kMixMaxImg), tile0 set
// here; sse indexed by out_index, the split map by blk0 + region.
template <int C16, int C8>
tx16_status mixed_bt_batch(const MixedParam* imgs, int n, unsigned long long* sse, uint8_t* split,
                           cudaStream_t stream) {
  using Cfg = MixCfg<C16>;
  MixedBtBatch<kMixMaxImg> P;
  P.nimg = n;
  P.sse = sse;
  P.split = split;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].p.tile0 = tiles;
    tiles += (imgs[i].p.nblk + kWarpTile - 1) / kWarpTile;
  }
  P.ntiles = tiles;
  auto kern = mixed_bt_kernel<kMixMaxImg, C16, C8>;
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::kSmem)) != cudaSuccess)
      return TX16_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Cfg::kThreads, Cfg::kSmem) != cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min((tiles + Cfg::kWarps - 1) / Cfg::kWarps, occ * device_sm_count()));
  kern<<<grid, Cfg::kThreads, Cfg::kSmem, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

}  // namespace tx16
