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
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "tx16_internal.h"
#include "tx16_net.cuh"
#include "tx16_pairnet.cuh"
#include "tx16_fused_common.cuh"

namespace tx16 {
namespace {

using namespace pairnet;

// Per-image state held in registers between image changes.
struct ImgState {
  const uint8_t* src;
  uint8_t* dst;
  int64_t sp, dp, blk0;
  int nbx, nblk, tile0, tile_end;
  unsigned magic;
  int out;  // index into sse[]
  bool quant;
  // column-task constants (column v of the task): scale by class e(u) = 0, 1, 2
  float2 fs[3];  // quantiser: sign_v * f ; no quantiser: sign_v * D'_u D'_v / 256
  float2 gg[3];  // g
  float2 gc[3];  // -2^23 g
  int h;         // kept rows in column v
};

__device__ __forceinline__ void load_image(const ImgParam* imgs, int nimg, int ntiles, int k, int v,
                                           ImgState& S) {
  const ImgParam& I = imgs[k];
  S.src = static_cast<const uint8_t*>(I.src);
  S.dst = static_cast<uint8_t*>(I.dst);
  S.sp = I.src_pitch;
  S.dp = I.dst_pitch;
  S.blk0 = I.blk0;
  S.nbx = I.nbx;
  S.nblk = I.nblk;
  S.tile0 = I.tile0;
  S.tile_end = (k + 1 < nimg) ? imgs[k + 1].tile0 : ntiles;
  S.magic = I.div_magic;
  S.out = I.out_index;
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

constexpr int kSlotWords = 36;  // one column slot: 16 float2 + 4 words of padding

// (image row, byte column) of row l of block blk; row -1 past the image's end
__device__ __forceinline__ int2 row_pos(unsigned magic, int nbx, int nblk, int blk, int l) {
  if (blk >= nblk) return make_int2(-1, 0);
  const int2 c = block_coords(magic, nbx, blk);
  return make_int2(c.x * 16 + l, c.y * 16);
}

__device__ __forceinline__ uint4 load_row(const uint8_t* base, int64_t pitch, int2 rc) {
  return rc.x >= 0 ? __ldcs(reinterpret_cast<const uint4*>(base + int64_t(rc.x) * pitch + rc.y))
                   : make_uint4(0, 0, 0, 0);
}

// Tile schedules.  StaticRange: a contiguous range per CTA (grid sized to the
// SMs).  Dynamic: CTAs take chunks of `chunk` tiles from a device counter of
// the work list, the next chunk claimed one chunk ahead so prefetching never
// stalls on the atomic.  Both are called uniformly by the whole CTA.
struct StaticRange {
  int t0, t1;
  __device__ __forceinline__ int first() const { return t0 < t1 ? t0 : -1; }
  __device__ __forceinline__ int next(int t) const { return t + 1 < t1 ? t + 1 : -1; }
};

struct DynamicChunks {
  unsigned* counter;
  int ntiles, chunk, cur_end, next_start;
  int* slot;  // shared-memory broadcast slot
  __device__ __forceinline__ int grab() {
    __syncthreads();
    if (threadIdx.x == 0) *slot = int(atomicAdd(counter, unsigned(chunk)));
    __syncthreads();
    return *slot;
  }
  __device__ __forceinline__ int first() {
    const int s = grab();
    if (s >= ntiles) return -1;
    cur_end = min(s + chunk, ntiles);
    next_start = grab();
    return s;
  }
  __device__ __forceinline__ int next(int t) {
    if (t + 1 < cur_end) return t + 1;
    const int s = next_start;
    if (s >= ntiles) return -1;
    cur_end = min(s + chunk, ntiles);
    next_start = grab();
    return s;
  }
};

// The fused codec over the tiles a schedule hands out.  imgs: descriptors of
// the launch (tile0 ascending), in parameter space or in a device work list.
template <class Z, bool LEV, bool DST, class Sched>
__device__ __forceinline__ void codec_tiles(const ImgParam* imgs, int nimg, int ntiles,
                                            unsigned long long* sse, int* levels, Sched& sched) {
  // column slots: slot p*V + v holds column v of block pair p (16 float2)
  __shared__ __align__(16) float smem[8 * Z::V * kSlotWords];
  constexpr int kTasks = 8 * Z::V;  // column tasks per tile
  const int l = threadIdx.x & 15;   // row of the block pair (row phases)
  const int p = threadIdx.x >> 4;   // block pair: blocks p and p + 8 of the tile
  const int task = threadIdx.x;     // column task: pair task / V, column task % V
  const int tv = task % Z::V;
  const bool col_active = task < kTasks;
  const bool warp_has_cols = (task & ~31) < kTasks;

  int t = sched.first();
  if (t < 0) return;
  int k = image_of_tile(imgs, nimg, t);
  ImgState S;
  load_image(imgs, nimg, ntiles, k, tv, S);
  unsigned long long acc = 0;

  // rows of the current tile (prefetched one tile ahead) and their positions
  uint4 ra, rb;
  int2 pa_next, pb_next;
  {
    const int base = (t - S.tile0) * kTileBlocks;
    pa_next = row_pos(S.magic, S.nbx, S.nblk, base + p, l);
    pb_next = row_pos(S.magic, S.nbx, S.nblk, base + p + 8, l);
    ra = load_row(S.src, S.sp, pa_next);
    rb = load_row(S.src, S.sp, pb_next);
  }

  while (t >= 0) {
    const int tn = sched.next(t);  // uniform over the CTA
    if (t < S.tile0 || t >= S.tile_end) {  // uniform: another image
      if (sse) flush_sse(sse, S.out, acc);
      acc = 0;
      k = image_of_tile(imgs, nimg, t);
      load_image(imgs, nimg, ntiles, k, tv, S);
    }
    const uint4 ca = ra, cb = rb;
    const int2 pa = pa_next, pb = pb_next;
    // prefetch the next tile's rows (they may belong to another image)
    if (tn >= 0) {
      if (tn >= S.tile0 && tn < S.tile_end) {  // same image: everything is in registers
        const int base = (tn - S.tile0) * kTileBlocks;
        pa_next = row_pos(S.magic, S.nbx, S.nblk, base + p, l);
        pb_next = row_pos(S.magic, S.nbx, S.nblk, base + p + 8, l);
        ra = load_row(S.src, S.sp, pa_next);
        rb = load_row(S.src, S.sp, pb_next);
      } else {  // uniform: the next tile starts another image
        const ImgParam& In = imgs[image_of_tile(imgs, nimg, tn)];
        const int base = (tn - In.tile0) * kTileBlocks;
        pa_next = row_pos(In.div_magic, In.nbx, In.nblk, base + p, l);
        pb_next = row_pos(In.div_magic, In.nbx, In.nblk, base + p + 8, l);
        ra = load_row(static_cast<const uint8_t*>(In.src), In.src_pitch, pa_next);
        rb = load_row(static_cast<const uint8_t*>(In.src), In.src_pitch, pb_next);
      }
    }

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
      for (int v = 0; v < Z::V; ++v)
        *reinterpret_cast<float2*>(&smem[(p * Z::V + v) * kSlotWords + 2 * l]) = y[v];
      if (LEV) {  // columns v >= V hold no kept coefficient: level 0 (row l of both blocks)
        const int base = (t - S.tile0) * kTileBlocks;
        int* ra_ = levels + (S.blk0 + base + p) * 256 + l * 16;
#pragma unroll
        for (int v = Z::V; v < 16; ++v) {
          if (pa.x >= 0) __stcs(ra_ + v, 0);
          if (pb.x >= 0) __stcs(ra_ + 8 * 256 + v, 0);
        }
      }
    }
    __syncthreads();

    // ---- column phase: task (pair task / V, column tv) ----
    if (warp_has_cols) {
      // lanes past the last task (a partly used warp) read slot 0 and write nothing
      float* slot = &smem[(col_active ? task : 0) * kSlotWords];
      float2 x[16];
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        const float4 q = *reinterpret_cast<const float4*>(slot + 2 * u);
        x[u] = make_float2(q.x, q.y);
        x[u + 1] = make_float2(q.z, q.w);
      }
      float2 n[16];
      Z::FwdCol::run(x, n);  // n[u] = FwdCol::sign(u) * (row-pass sign of tv) * Y[u][tv]
      float2 w[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) w[u] = make_float2(0.f, 0.f);
      const int tp = task / Z::V;
      const int tbase = (t - S.tile0) * kTileBlocks;
      const bool tva = col_active && tbase + tp < S.nblk;
      const bool tvb = col_active && tbase + tp + 8 < S.nblk;
      int* lev_a = LEV ? levels + (S.blk0 + tbase + tp) * 256 + tv : nullptr;
      int* lev_b = LEV ? lev_a + 8 * 256 : nullptr;
      if (S.quant) {
#pragma unroll
        for (int u = 0; u < Z::U; ++u) {
          const int e = scale_class(u);
          const float2 tq = __fmul2_rn(n[u], S.fs[e]);
          const float2 a = make_float2(fabsf(tq.x), fabsf(tq.y));
          const float2 m = __fadd2_rd(__fadd2_rd(a, f2(0.5f)), f2(8388608.f));  // 2^23 + floor(|t| + 1/2)
          float2 q = __ffma2_rn(m, S.gg[e], S.gc[e]);                          // fl32(level * g)
          q.x = __uint_as_float(__float_as_uint(q.x) | (__float_as_uint(tq.x) & 0x80000000u));
          q.y = __uint_as_float(__float_as_uint(q.y) | (__float_as_uint(tq.y) & 0x80000000u));
          const bool keep = u < S.h;
          w[u] = keep ? q : make_float2(0.f, 0.f);
          if (LEV) {
            // level = sign(FwdCol) * sign(t) * floor(|t| + 1/2)
            const unsigned flip = Z::FwdCol::sign(u) < 0 ? 1u : 0u;
            int la = int(__float_as_uint(m.x) - 0x4B000000u), lb = int(__float_as_uint(m.y) - 0x4B000000u);
            la = ((__float_as_uint(tq.x) >> 31) != flip) ? -la : la;
            lb = ((__float_as_uint(tq.y) >> 31) != flip) ? -lb : lb;
            if (tva) __stcs(lev_a + u * 16, keep ? la : 0);
            if (tvb) __stcs(lev_b + u * 16, keep ? lb : 0);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < Z::U; ++u) {
          const float2 q = __fmul2_rn(n[u], S.fs[scale_class(u)]);
          const bool keep = u < S.h;
          w[u] = keep ? q : make_float2(0.f, 0.f);
          if (LEV) {
            const float sgn = float(Z::FwdCol::sign(u)) * (((kFwdNegMask >> tv) & 1u) ? -1.f : 1.f);
            if (tva) __stcs(lev_a + u * 16, keep ? __float2int_rn(sgn * n[u].x) : 0);
            if (tvb) __stcs(lev_b + u * 16, keep ? __float2int_rn(sgn * n[u].y) : 0);
          }
        }
      }
      if (LEV) {
#pragma unroll
        for (int u = Z::U; u < 16; ++u) {
          if (tva) __stcs(lev_a + u * 16, 0);
          if (tvb) __stcs(lev_b + u * 16, 0);
        }
      }
      float2 z[16];
      Z::InvCol::run(w, z);  // z[i] = (T^t W)[i][tv]
      if (col_active) {
#pragma unroll
        for (int i = 0; i < 16; i += 2)
          *reinterpret_cast<float4*>(slot + 2 * i) = make_float4(z[i].x, z[i].y, z[i + 1].x, z[i + 1].y);
      }
    }
    __syncthreads();

    // ---- row phase: inverse row transform, rounding, store, SSE ----
    {
      float2 w[16];
#pragma unroll
      for (int v = 0; v < 16; ++v)
        w[v] = v < Z::V ? *reinterpret_cast<const float2*>(&smem[(p * Z::V + v) * kSlotWords + 2 * l])
                        : make_float2(0.f, 0.f);
      float2 z[16];
      Z::InvRow::run(w, z);  // z[j] = sign[j] * X_tilde[l][j]
      // sample = clip(floor(X + 1/2), 0, 255): the bits of
      // RD(RD(X + 1/2) 2^-149), clamped and packed four to a word
      int na[16], nb[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 r = Z::InvRow::sign(j) >= 0 ? __fadd2_rd(z[j], f2(0.5f)) : sub2_rd(f2(0.5f), z[j]);
        const float2 n = floor_bits2(r);
        na[j] = __float_as_int(n.x);
        nb[j] = __float_as_int(n.y);
      }
      unsigned xa[4], xb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xa[q] = pack4_sat_u8(na[4 * q], na[4 * q + 1], na[4 * q + 2], na[4 * q + 3]);
        xb[q] = pack4_sat_u8(nb[4 * q], nb[4 * q + 1], nb[4 * q + 2], nb[4 * q + 3]);
      }
      if (DST) {
        if (pa.x >= 0)
          __stcs(reinterpret_cast<uint4*>(S.dst + int64_t(pa.x) * S.dp + pa.y), make_uint4(xa[0], xa[1], xa[2], xa[3]));
        if (pb.x >= 0)
          __stcs(reinterpret_cast<uint4*>(S.dst + int64_t(pb.x) * S.dp + pb.y), make_uint4(xb[0], xb[1], xb[2], xb[3]));
      }
      // SSE = sum |x - y|^2 over the row's bytes (vabsdiff4, then dp4a).  A
      // block past the end of the image was loaded as zeros and reconstructs
      // to zeros, so it adds nothing.
      const unsigned ia[4] = {ca.x, ca.y, ca.z, ca.w}, ib[4] = {cb.x, cb.y, cb.z, cb.w};
      unsigned s1 = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned da = __vabsdiffu4(ia[q], xa[q]), db = __vabsdiffu4(ib[q], xb[q]);
        s1 = __dp4a(da, da, s1);
        s1 = __dp4a(db, db, s1);
      }
      acc += s1;
    }
    t = tn;
  }
  if (sse) flush_sse(sse, S.out, acc);
}

// By-value launch: descriptors in the kernel parameters, a static tile range
// per CTA.  MAXI images per launch, zone class Z, LEV = write levels, DST =
// write reconstructed samples.
template <int MAXI, class Z, bool LEV, bool DST>
__global__ void __launch_bounds__(128, Z::kMinCtas) fused_u8_kernel(const __grid_constant__ BatchParams<MAXI> P) {
  const int per = (P.ntiles + gridDim.x - 1) / gridDim.x;
  StaticRange sched{int(blockIdx.x) * per, min(int(blockIdx.x) * per + per, P.ntiles)};
  codec_tiles<Z, LEV, DST>(P.img, P.nimg, P.ntiles, P.sse, P.coeffs, sched);
}

// Work-list launch: descriptors in device memory, tiles handed out in chunks
// from a device counter (reset to 0 before the launch).
template <class Z, bool LEV, bool DST>
__global__ void __launch_bounds__(128, Z::kMinCtas)
    fused_u8_list_kernel(const ImgParam* __restrict__ imgs, int nimg, int ntiles, unsigned* counter, int chunk,
                         unsigned long long* sse, int* levels) {
  __shared__ int slot;
  DynamicChunks sched{counter, ntiles, chunk, 0, 0, &slot};
  codec_tiles<Z, LEV, DST>(imgs, nimg, ntiles, sse, levels, sched);
}

template <int MAXI, class Z, bool LEV, bool DST>
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
    P.img[i].out_index = i;
    tiles += (imgs[i].nblk + kTileBlocks - 1) / kTileBlocks;
  }
  P.ntiles = tiles;
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    // prefer shared memory over L1 so the register limit, not the carveout,
    // sets the resident CTAs per SM
    cudaFuncSetAttribute(fused_u8_kernel<MAXI, Z, LEV, DST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fused_u8_kernel<MAXI, Z, LEV, DST>, 128, 0) !=
            cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min(tiles, occ * device_sm_count()));
  fused_u8_kernel<MAXI, Z, LEV, DST><<<grid, 128, 0, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

template <int MAXI, bool LEV, bool DST>
tx16_status launch_fused_zone(int zone, const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                              cudaStream_t stream) {
  switch (zone) {
    case 0: return launch_fused<MAXI, ZoneA, LEV, DST>(imgs, n, sse, levels, stream);
    case 1: return launch_fused<MAXI, ZoneB, LEV, DST>(imgs, n, sse, levels, stream);
    case 2: return launch_fused<MAXI, ZoneC, LEV, DST>(imgs, n, sse, levels, stream);
    case 3: return launch_fused<MAXI, ZoneD, LEV, DST>(imgs, n, sse, levels, stream);
    default: return launch_fused<MAXI, ZoneE, LEV, DST>(imgs, n, sse, levels, stream);
  }
}

template <int MAXI>
tx16_status launch_fused_modes(int zone, const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                               cudaStream_t stream) {
  const bool dst = imgs[0].dst != nullptr;
  // no level output: one block per thread in registers -- unless the batch has fewer 32-block warp tiles than the GPU
  // has SMs: then each warp would code a single tile, a whole block per
  // thread in series, and the pair kernel (16 blocks over 128 threads) ends
  // sooner
  int64_t blocks = 0;
  for (int i = 0; i < n; ++i) blocks += imgs[i].nblk;
  const bool small = (blocks + 31) / 32 < int64_t(device_sm_count());
  if (!small && fused_bt_supports(zone, levels != nullptr)) return launch_fused_bt(zone, dst, imgs, n, sse, stream);
  if (levels != nullptr)
    return dst ? launch_fused_zone<MAXI, true, true>(zone, imgs, n, sse, levels, stream)
               : launch_fused_zone<MAXI, true, false>(zone, imgs, n, sse, levels, stream);
  return dst ? launch_fused_zone<MAXI, false, true>(zone, imgs, n, sse, levels, stream)
             : launch_fused_zone<MAXI, false, false>(zone, imgs, n, sse, levels, stream);
}

template <class Z, bool LEV, bool DST>
int list_max_ctas() {
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    cudaFuncSetAttribute(fused_u8_list_kernel<Z, LEV, DST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fused_u8_list_kernel<Z, LEV, DST>, 128, 0) !=
            cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}

template <class Z, bool LEV, bool DST>
tx16_status launch_list(const ImgParam* d_imgs, int nimg, int ntiles, unsigned* counter, int chunk, int ctas_per_sm,
                        unsigned long long* sse, int32_t* levels, cudaStream_t stream) {
  const int occ = list_max_ctas<Z, LEV, DST>();
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  const int grid = std::max(1, std::min((ntiles + chunk - 1) / chunk, per_sm * device_sm_count()));
  fused_u8_list_kernel<Z, LEV, DST><<<grid, 128, 0, stream>>>(d_imgs, nimg, ntiles, counter, chunk, sse, levels);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

template <class Z>
tx16_status launch_list_modes(bool lev, bool dst, const ImgParam* d_imgs, int nimg, int ntiles, unsigned* counter,
                              int chunk, int ctas_per_sm, unsigned long long* sse, int32_t* levels,
                              cudaStream_t stream) {
  if (lev)
    return dst ? launch_list<Z, true, true>(d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream)
               : launch_list<Z, true, false>(d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
  return dst ? launch_list<Z, false, true>(d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream)
             : launch_list<Z, false, false>(d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
}

template <class Z>
int list_max_ctas_modes(bool lev, bool dst) {
  if (lev) return dst ? list_max_ctas<Z, true, true>() : list_max_ctas<Z, true, false>();
  return dst ? list_max_ctas<Z, false, true>() : list_max_ctas<Z, false, false>();
}

}  // namespace

tx16_status launch_fused_list(int zone, bool lev, bool dst, const ImgParam* d_imgs, int nimg, int ntiles,
                              unsigned* counter, int chunk, int ctas_per_sm, unsigned long long* sse,
                              int32_t* levels, cudaStream_t stream) {
  switch (zone) {
    case 0: return launch_list_modes<ZoneA>(lev, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
    case 1: return launch_list_modes<ZoneB>(lev, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
    case 2: return launch_list_modes<ZoneC>(lev, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
    case 3: return launch_list_modes<ZoneD>(lev, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
    default: return launch_list_modes<ZoneE>(lev, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, levels, stream);
  }
}

int fused_list_max_ctas(int zone, bool lev, bool dst) {
  switch (zone) {
    case 0: return list_max_ctas_modes<ZoneA>(lev, dst);
    case 1: return list_max_ctas_modes<ZoneB>(lev, dst);
    case 2: return list_max_ctas_modes<ZoneC>(lev, dst);
    case 3: return list_max_ctas_modes<ZoneD>(lev, dst);
    default: return list_max_ctas_modes<ZoneE>(lev, dst);
  }
}

bool fused_eligible(const ImgParam& p) {
  const int bits = p.flags & 0xff;
  return bits == 8 && (!(p.flags & kQuantFlag) || p.g[0] * 16.0f >= kFusedMinQ);
}

// Smallest zonal class covering every image of the launch: class c holds the
// zones inside Z_rmax(c) (r_max = 8, 16, 32, 64, 128, 256), compared column by
// column (zig-zag zones nest, so this is the class of the largest r).  The
// pair kernel codes classes 4 and 5 with the full 16 x 16 networks.
int fused_zone_class(const ImgParam* imgs, int n) {
  static const struct Heights {
    uint8_t h[6][16];
    Heights() {
      for (int c = 0; c < 6; ++c) zonal_column_heights(bt_class_rmax(c), h[c]);
    }
  } H;
  uint8_t need[16] = {};
  for (int i = 0; i < n; ++i)
    for (int v = 0; v < 16; ++v) need[v] = std::max(need[v], imgs[i].colh[v]);
  for (int c = 0; c < 5; ++c) {
    bool in = true;
    for (int v = 0; v < 16; ++v) in = in && need[v] <= H.h[c][v];
    if (in) return c;
  }
  return 5;
}

tx16_status launch_fused_u8(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                            cudaStream_t stream) {
  // Without levels, a batch whose images fall in different zonal classes
  // runs as one launch per class on the one-block-per-thread kernel, each
  // image adding into its own SSE slot: coded in chunks by position, every
  // image of a chunk would run at the chunk's largest class.
  if (levels == nullptr && n > 1) {
    std::vector<int> cls(n);
    bool mixed = false;
    int64_t blocks = 0;
    bool all_bt = true;  // every class present runs on the one-block-per-thread kernel
    for (int i = 0; i < n; ++i) {
      cls[i] = fused_zone_class(&imgs[i], 1);
      mixed = mixed || cls[i] != cls[0];
      all_bt = all_bt && fused_bt_supports(cls[i], false);
      blocks += imgs[i].nblk;
    }
    const bool dst = imgs[0].dst != nullptr;
    if (mixed && all_bt && (blocks + 31) / 32 >= int64_t(device_sm_count())) {
      std::vector<ImgParam> g;
      for (int c = 0; c < 6; ++c) {
        g.clear();
        for (int i = 0; i < n; ++i) {
          if (cls[i] != c) continue;
          ImgParam p = imgs[i];
          p.out_index = i;
          g.push_back(p);
        }
        for (size_t s = 0; s < g.size(); s += kMaxImg) {
          const int m = int(std::min<size_t>(kMaxImg, g.size() - s));
          const tx16_status st = launch_fused_bt_grouped(c, dst, g.data() + s, m, sse, stream);
          if (st != TX16_OK) return st;
        }
      }
      return TX16_OK;
    }
  }
  for (int s = 0; s < n; s += kMaxImg) {
    const int m = std::min(kMaxImg, n - s);
    const int zone = fused_zone_class(imgs + s, m);
    const tx16_status st = m <= 8 ? launch_fused_modes<8>(zone, imgs + s, m, sse ? sse + s : nullptr, levels, stream)
                                  : launch_fused_modes<kMaxImg>(zone, imgs + s, m, sse ? sse + s : nullptr, levels,
                                                                stream);
    if (st != TX16_OK) return st;
  }
  return TX16_OK;
}

}  // namespace tx16
