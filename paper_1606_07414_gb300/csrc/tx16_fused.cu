// Fused codec for 8-bit planes: forward transform, S-merged quantiser, inverse,
// reconstruction and squared error of every 16x16 block in one pass.
//
// Mapping.  A CTA of 128 threads works on a tile of 16 consecutive blocks of
// one image.  Half-warp p (p = 0..7) owns the block PAIR (p, p + 8) of the
// tile, and every value it handles is a float2 (block p, block p + 8), so the
// Blackwell packed-FP32 instructions (__fadd2_rn, __ffma2_rn, __fmul2_rn,
// __fadd2_rd) do two blocks' arithmetic per instruction.
//   row phase     thread l: row l of both blocks -> forward row transform
//   column phase  thread v: column v of both blocks -> forward column
//                 transform, quantiser, inverse column transform
//   row phase     thread l: inverse row transform, rounding, store, SSE
// Row/column exchanges go through a 16 x 36-word shared buffer per pair.
//
// Exactness.  The forward transform runs in binary32 on integers below 2^24,
// so it is exact (Y = T X T^t bit for bit).  The quantiser and the inverse
// follow the binary32 definition of the library exactly:
//   level = round_half_away(fl32(Y * f)),  f = fl32(s_u s_v / q)
//   W     = fl32(level * g),               g = fl32(q s_u s_v)
//   T^t W T through the transposed factorisation, columns first
// and with no quantiser the inverse is exact as well (values k / 256 with
// |k| < 2^24).  The networks come from tx16_pairnet.cuh (generated), where
// negations are folded into the additions at compile time and the zonal
// extents prune the work.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "tx16_internal.h"
#include "tx16_net.cuh"
#include "tx16_pairnet.cuh"

namespace tx16 {
namespace {

using namespace pairnet;

template <int U_, int V_, class FR, class FC, class IC, class IR>
struct Zone {
  static constexpr int U = U_;  // kept rows u < U
  static constexpr int V = V_;  // kept columns v < V
  using FwdRow = FR;
  using FwdCol = FC;
  using InvCol = IC;
  using InvRow = IR;
};
using ZoneA = Zone<3, 4, FwdRow4, FwdCol3, InvCol3, InvRow4>;        // r <= 8
using ZoneB = Zone<5, 6, FwdRow6, FwdCol5, InvCol5, InvRow6>;        // r <= 16
using ZoneC = Zone<7, 8, FwdRow8, FwdCol7, InvCol7, InvRow8>;        // r <= 32
using ZoneD = Zone<11, 10, FwdRow10, FwdCol11, InvCol11, InvRow10>;  // r <= 64
using ZoneE = Zone<16, 16, FwdRow16, FwdCol16, InvCol16, InvRow16>;  // any r

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

// Per-image state held in registers between image changes.
struct ImgState {
  const uint8_t* src;
  uint8_t* dst;
  int64_t sp, dp, blk0;
  int nbx, nblk, tile0, tile_end;
  unsigned magic;
  int shift;
  bool quant;
  // column-thread constants (column v = l): scale by class e(u) = 0, 1, 2
  float2 fs[3];  // quantiser: sign_v * f ; no quantiser: sign_v * D'_u D'_v / 256
  float2 gg[3];  // g
  float2 gc[3];  // -2^23 g
  int h;         // kept rows in column v
};

template <int MAXI>
__device__ __forceinline__ void load_image(const BatchParams<MAXI>& P, int k, int v, ImgState& S) {
  const ImgParam& I = P.img[k];
  S.src = static_cast<const uint8_t*>(I.src);
  S.dst = static_cast<uint8_t*>(I.dst);
  S.sp = I.src_pitch;
  S.dp = I.dst_pitch;
  S.blk0 = I.blk0;
  S.nbx = I.nbx;
  S.nblk = I.nblk;
  S.tile0 = I.tile0;
  S.tile_end = (k + 1 < P.nimg) ? P.img[k + 1].tile0 : P.ntiles;
  S.magic = I.div_magic;
  S.shift = I.div_shift;
  S.quant = (I.flags & kQuantFlag) != 0;
  const int ev = scale_class(v);
  const float sv = ((kFwdNegMask >> v) & 1u) ? -1.f : 1.f;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (S.quant) {
      S.fs[e] = f2(sv * I.f[e + ev]);
      S.gg[e] = f2(I.g[e + ev]);
      S.gc[e] = f2(-8388608.f * I.g[e + ev]);
    } else {
      S.fs[e] = f2(sv * float(1 << (e + ev)) * (1.f / 256.f));
      S.gg[e] = f2(0.f);
      S.gc[e] = f2(0.f);
    }
  }
  S.h = I.colh[v];
}

__device__ __forceinline__ void block_coords(const ImgState& S, int blk, int& by, int& bx) {
  unsigned q = __umulhi(unsigned(blk), S.magic) >> S.shift;
  int r = blk - int(q) * S.nbx;
  if (r >= S.nbx) {
    ++q;
    r -= S.nbx;
  }
  by = int(q);
  bx = r;
}

__device__ __forceinline__ void flush_sse(unsigned long long* sse, int img, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicAdd(sse + img, v);
}

constexpr int kRowWords = 36;  // 16 float2 + 4 words of padding per row

template <int MAXI, class Z>
__global__ void __launch_bounds__(128) fused_u8_kernel(const __grid_constant__ BatchParams<MAXI> P) {
  __shared__ __align__(16) float smem[8][16][kRowWords];
  const int l = threadIdx.x & 15;  // row (row phases) or column v (column phase)
  const int p = threadIdx.x >> 4;  // block pair: blocks p and p + 8 of the tile
  float(*Sm)[kRowWords] = smem[p];

  const int per = (P.ntiles + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per;
  const int t1 = min(t0 + per, P.ntiles);
  if (t0 >= t1) return;

  int k = 0;
  {
    int hi = P.nimg - 1;
    while (k < hi) {
      const int mid = (k + hi + 1) >> 1;
      if (P.img[mid].tile0 <= t0) k = mid; else hi = mid - 1;
    }
  }
  ImgState S;
  load_image(P, k, l, S);
  unsigned long long acc = 0;

  // rows of the current tile, prefetched one tile ahead
  uint4 ra = make_uint4(0, 0, 0, 0), rb = ra;
  auto row_ptrs = [&](const ImgState& s, int t, const uint8_t*& pa, const uint8_t*& pb) {
    const int base = (t - s.tile0) * kTileBlocks;
    int by, bx;
    pa = nullptr;
    pb = nullptr;
    if (base + p < s.nblk) {
      block_coords(s, base + p, by, bx);
      pa = s.src + (int64_t(by) * 16 + l) * s.sp + int64_t(bx) * 16;
    }
    if (base + p + 8 < s.nblk) {
      block_coords(s, base + p + 8, by, bx);
      pb = s.src + (int64_t(by) * 16 + l) * s.sp + int64_t(bx) * 16;
    }
  };
  {
    const uint8_t *pa, *pb;
    row_ptrs(S, t0, pa, pb);
    if (pa) ra = __ldcs(reinterpret_cast<const uint4*>(pa));
    if (pb) rb = __ldcs(reinterpret_cast<const uint4*>(pb));
  }

  for (int t = t0; t < t1; ++t) {
    if (t >= S.tile_end) {  // uniform: next image
      if (P.sse) flush_sse(P.sse, k, acc);
      acc = 0;
      while (t >= S.tile_end) {
        ++k;
        S.tile_end = (k + 1 < P.nimg) ? P.img[k + 1].tile0 : P.ntiles;
      }
      load_image(P, k, l, S);
    }
    const uint4 ca = ra, cb = rb;
    // prefetch the next tile's rows (possibly of the next image)
    if (t + 1 < t1) {
      const uint8_t *pa, *pb;
      if (t + 1 < S.tile_end) {
        row_ptrs(S, t + 1, pa, pb);
      } else {
        int kn = k;
        while (kn + 1 < P.nimg && P.img[kn + 1].tile0 <= t + 1) ++kn;
        ImgState Sn;
        const ImgParam& In = P.img[kn];
        Sn.src = static_cast<const uint8_t*>(In.src);
        Sn.sp = In.src_pitch;
        Sn.nbx = In.nbx;
        Sn.nblk = In.nblk;
        Sn.tile0 = In.tile0;
        Sn.magic = In.div_magic;
        Sn.shift = In.div_shift;
        row_ptrs(Sn, t + 1, pa, pb);
      }
      ra = pa ? __ldcs(reinterpret_cast<const uint4*>(pa)) : make_uint4(0, 0, 0, 0);
      rb = pb ? __ldcs(reinterpret_cast<const uint4*>(pb)) : make_uint4(0, 0, 0, 0);
    }
    const int base = (t - S.tile0) * kTileBlocks;
    const bool va = base + p < S.nblk;
    const bool vb = base + p + 8 < S.nblk;

    // ---- row phase: forward transform of row l of both blocks ----
    {
      const unsigned wa[4] = {ca.x, ca.y, ca.z, ca.w};
      const unsigned wb[4] = {cb.x, cb.y, cb.z, cb.w};
      float2 X[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) X[j] = make_float2(biased(wa[j >> 2], j & 3), biased(wb[j >> 2], j & 3));
      float2 y[16];
      Z::FwdRow::run(X, y);
#pragma unroll
      for (int v = 0; v < Z::V; v += 2)
        *reinterpret_cast<float4*>(&Sm[l][2 * v]) = make_float4(y[v].x, y[v].y, y[v + 1].x, y[v + 1].y);
    }
    __syncwarp();

    // ---- column phase: thread v = l ----
    {
      float2 x[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) x[u] = *reinterpret_cast<const float2*>(&Sm[u][2 * l]);
      float2 n[16];
      Z::FwdCol::run(x, n);  // n[u] = FwdCol::sign(u) * (row-pass sign of v) * Y[u][v]
      float2 w[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) w[u] = make_float2(0.f, 0.f);
      int* lev = P.coeffs;
      if (S.quant) {
#pragma unroll
        for (int u = 0; u < Z::U; ++u) {
          const int e = scale_class(u);
          const float2 t = __fmul2_rn(n[u], S.fs[e]);
          const float2 a = make_float2(fabsf(t.x), fabsf(t.y));
          const float2 m = __fadd2_rd(__fadd2_rd(a, f2(0.5f)), f2(8388608.f));  // 2^23 + floor(|t| + 1/2)
          float2 q = __ffma2_rn(m, S.gg[e], S.gc[e]);                          // fl32(level * g)
          q.x = __uint_as_float(__float_as_uint(q.x) | (__float_as_uint(t.x) & 0x80000000u));
          q.y = __uint_as_float(__float_as_uint(q.y) | (__float_as_uint(t.y) & 0x80000000u));
          if (u < S.h) w[u] = q;
          if (lev != nullptr) {
            // level = sign(FwdCol) * sign(t) * floor(|t| + 1/2)
            int la = int(__float_as_uint(m.x) - 0x4B000000u), lb = int(__float_as_uint(m.y) - 0x4B000000u);
            if ((__float_as_uint(t.x) >> 31) != (Z::FwdCol::sign(u) < 0 ? 1u : 0u)) la = -la;
            if ((__float_as_uint(t.y) >> 31) != (Z::FwdCol::sign(u) < 0 ? 1u : 0u)) lb = -lb;
            if (u >= S.h) la = lb = 0;
            if (va) __stcs(lev + (S.blk0 + base + p) * 256 + u * 16 + l, la);
            if (vb) __stcs(lev + (S.blk0 + base + p + 8) * 256 + u * 16 + l, lb);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < Z::U; ++u) {
          const float2 q = __fmul2_rn(n[u], S.fs[scale_class(u)]);
          if (u < S.h) w[u] = q;
          if (lev != nullptr) {
            const float sgn = float(Z::FwdCol::sign(u)) * (((kFwdNegMask >> l) & 1u) ? -1.f : 1.f);
            const int la = u < S.h ? __float2int_rn(sgn * n[u].x) : 0;
            const int lb = u < S.h ? __float2int_rn(sgn * n[u].y) : 0;
            if (va) __stcs(lev + (S.blk0 + base + p) * 256 + u * 16 + l, la);
            if (vb) __stcs(lev + (S.blk0 + base + p + 8) * 256 + u * 16 + l, lb);
          }
        }
      }
      if (lev != nullptr) {
#pragma unroll
        for (int u = Z::U; u < 16; ++u) {
          if (va) __stcs(lev + (S.blk0 + base + p) * 256 + u * 16 + l, 0);
          if (vb) __stcs(lev + (S.blk0 + base + p + 8) * 256 + u * 16 + l, 0);
        }
      }
      float2 z[16];
      Z::InvCol::run(w, z);  // z[i] = (T^t W)[i][v]
#pragma unroll
      for (int i = 0; i < 16; ++i) *reinterpret_cast<float2*>(&Sm[i][2 * l]) = z[i];
    }
    __syncwarp();

    // ---- row phase: inverse row transform, rounding, store, SSE ----
    {
      float2 w[16];
#pragma unroll
      for (int v = 0; v < 16; ++v) w[v] = make_float2(0.f, 0.f);
#pragma unroll
      for (int v = 0; v < Z::V; v += 2) {
        const float4 q = *reinterpret_cast<const float4*>(&Sm[l][2 * v]);
        w[v] = make_float2(q.x, q.y);
        w[v + 1] = make_float2(q.z, q.w);
      }
      float2 z[16];
      Z::InvRow::run(w, z);  // z[j] = sign[j] * X_tilde[l][j]
      // sample = clip(floor(X + 1/2), 0, 255): the low byte of the binary16
      // value RZ(RD(X + 1024.5)) clamped to [1024, 1279]
      unsigned h[16];
      const __half2 lo = __float2half2_rn(1024.f), hi = __float2half2_rn(1279.f);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 r = Z::InvRow::sign(j) >= 0 ? __fadd2_rd(z[j], f2(1024.5f))
                                                 : __ffma2_rd(z[j], pm1(), f2(1024.5f));
        __half2 hv;
        const unsigned raw = cvt_rz_h2(r);
        hv = *reinterpret_cast<const __half2*>(&raw);
        hv = __hmin2(__hmax2(hv, lo), hi);
        h[j] = *reinterpret_cast<const unsigned*>(&hv);
      }
      unsigned oa[4], ob[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned t01 = __byte_perm(h[4 * q], h[4 * q + 1], 0x6240u);
        const unsigned t23 = __byte_perm(h[4 * q + 2], h[4 * q + 3], 0x6240u);
        oa[q] = __byte_perm(t01, t23, 0x5410u);
        ob[q] = __byte_perm(t01, t23, 0x7632u);
      }
      if (S.dst != nullptr) {
        int by, bx;
        if (va) {
          block_coords(S, base + p, by, bx);
          __stcs(reinterpret_cast<uint4*>(S.dst + (int64_t(by) * 16 + l) * S.dp + int64_t(bx) * 16),
                 make_uint4(oa[0], oa[1], oa[2], oa[3]));
        }
        if (vb) {
          block_coords(S, base + p + 8, by, bx);
          __stcs(reinterpret_cast<uint4*>(S.dst + (int64_t(by) * 16 + l) * S.dp + int64_t(bx) * 16),
                 make_uint4(ob[0], ob[1], ob[2], ob[3]));
        }
      }
      // SSE = sum x^2 + sum y^2 - 2 sum x y over the row's bytes (dp4a)
      const unsigned ia[4] = {ca.x, ca.y, ca.z, ca.w}, ib[4] = {cb.x, cb.y, cb.z, cb.w};
      unsigned sxx = 0, syy = 0, sxy = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (va) {
          sxx = __dp4a(ia[q], ia[q], sxx);
          syy = __dp4a(oa[q], oa[q], syy);
          sxy = __dp4a(ia[q], oa[q], sxy);
        }
        if (vb) {
          sxx = __dp4a(ib[q], ib[q], sxx);
          syy = __dp4a(ob[q], ob[q], syy);
          sxy = __dp4a(ib[q], ob[q], sxy);
        }
      }
      acc += (unsigned long long)(sxx + syy - 2u * sxy);
    }
  }
  if (P.sse) flush_sse(P.sse, k, acc);
}

template <int MAXI, class Z>
tx16_status launch_fused(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                         cudaStream_t stream) {
  BatchParams<MAXI> P;
  P.nimg = n;
  P.sse = sse;
  P.coeffs = levels;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].tile0 = tiles;
    tiles += (imgs[i].nblk + kTileBlocks - 1) / kTileBlocks;
  }
  P.ntiles = tiles;
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fused_u8_kernel<MAXI, Z>, 128, 0) != cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min(tiles, occ * device_sm_count()));
  fused_u8_kernel<MAXI, Z><<<grid, 128, 0, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

template <int MAXI>
tx16_status launch_fused_zone(int zone, const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                              cudaStream_t stream) {
  switch (zone) {
    case 0: return launch_fused<MAXI, ZoneA>(imgs, n, sse, levels, stream);
    case 1: return launch_fused<MAXI, ZoneB>(imgs, n, sse, levels, stream);
    case 2: return launch_fused<MAXI, ZoneC>(imgs, n, sse, levels, stream);
    case 3: return launch_fused<MAXI, ZoneD>(imgs, n, sse, levels, stream);
    default: return launch_fused<MAXI, ZoneE>(imgs, n, sse, levels, stream);
  }
}

}  // namespace

// Smallest zone class covering every image of the launch (extents of Z_r).
int fused_zone_class(const ImgParam* imgs, int n) {
  int U = 0, V = 0;
  for (int i = 0; i < n; ++i)
    for (int v = 0; v < 16; ++v)
      if (imgs[i].colh[v] > 0) {
        U = std::max(U, int(imgs[i].colh[v]));
        V = std::max(V, v + 1);
      }
  const int cu[4] = {3, 5, 7, 11}, cv[4] = {4, 6, 8, 10};
  for (int c = 0; c < 4; ++c)
    if (U <= cu[c] && V <= cv[c]) return c;
  return 4;
}

tx16_status launch_fused_u8(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                            cudaStream_t stream) {
  for (int s = 0; s < n; s += kMaxImg) {
    const int m = std::min(kMaxImg, n - s);
    const int zone = fused_zone_class(imgs + s, m);
    const tx16_status st = m <= 8 ? launch_fused_zone<8>(zone, imgs + s, m, sse ? sse + s : nullptr, levels, stream)
                                  : launch_fused_zone<kMaxImg>(zone, imgs + s, m, sse ? sse + s : nullptr, levels,
                                                               stream);
    if (st != TX16_OK) return st;
  }
  return TX16_OK;
}

}  // namespace tx16
