// Mixed 8/16 tiling (tx16_codec_mixed): the video experiment's second
// scenario (Sec. 3.2), where the 8-point approximation T8 (14 additions,
// Sec. 2.1) and the 16-point T code blocks side by side.  Every 16x16 region
// is coded both ways -- one 16x16 block with T, or four 8x8 blocks with T8 --
// and the tiling with the smaller squared error is kept (ties: 16x16), or one
// tiling is forced.
//
// Mapping: 16 threads per region, thread l holding row l; 16 regions per CTA.
// The 16-point path is the general kernel's (int32 forward, binary32 or exact
// inverse, tx16_block.cuh).  The 8-point path runs on the same rows: the two
// 8-sample halves of row l through T8, an exchange through shared memory,
// then thread v transforms column v of the upper and of the lower 8x8 block.
// Quantiser for 8x8 blocks (S8 merged, Sec. 2.1 applied to T8):
//   level = round_half_away(fl32(fl32(Y8) * f8)), f8 = fl32(s8_u s8_v / q),
//   W = fl32(level * g8), g8 = fl32(q s8_u s8_v), s8_u s8_v = 2^(-3 + k/2),
//   k = c(u) + c(v), c = (0, 2, 1, 2, 0, 2, 1, 2);
// without a quantiser 64 X_tilde = T8^t (D8 Y8 D8) T8 exactly, D8 = 2^c.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "tx16_block.cuh"
#include "tx16_internal.h"
#include "tx16_net.cuh"

namespace tx16 {
ImgParam make_param(const tx16_image& in, const tx16_image* out, const tx16_qparams& qp, int64_t blk0);

namespace {

template <int MAXI>
struct MixedBatch {
  int32_t nimg, ntiles;
  unsigned long long* sse;  // indexed by out_index
  uint8_t* split;
  MixedParam img[MAXI];
};
static_assert(sizeof(MixedBatch<kMixMaxImg>) < 32000, "kernel parameters too large");

__device__ __forceinline__ int c8(int u) { return (u & 1) ? 2 : ((u & 2) ? 1 : 0); }  // 0,2,1,2,0,2,1,2

__device__ __forceinline__ int round_div64(int n) { return n >= 0 ? (n + 32) >> 6 : -((32 - n) >> 6); }

template <typename Smp, int MAXI>
__global__ void __launch_bounds__(kThreads) mixed_kernel(const __grid_constant__ MixedBatch<MAXI> P) {
  __shared__ int sm16[kTileBlocks][16][17];
  __shared__ int sm8[kTileBlocks][16][17];
  const int l = threadIdx.x & 15;
  const int b = threadIdx.x >> 4;
  int(*S)[17] = sm16[b];
  int(*S8)[17] = sm8[b];
  using IO = RowIO<Smp>;
  const int per = (P.ntiles + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per;
  const int t1 = min(t0 + per, P.ntiles);
  if (t0 >= t1) return;
  int k = 0;
  while (k + 1 < P.nimg && P.img[k + 1].p.tile0 <= t0) ++k;
  unsigned long long acc = 0;
  int acc_img = k;
  for (int t = t0; t < t1; ++t) {
    while (k + 1 < P.nimg && P.img[k + 1].p.tile0 <= t) ++k;  // uniform
    if (k != acc_img) {
      if (P.sse) flush_sse_rows(P.sse, P.img[acc_img].p.out_index, acc);
      acc = 0;
      acc_img = k;
    }
    const MixedParam& M = P.img[k];
    const ImgParam& I = M.p;
    const int blk = (t - I.tile0) * kTileBlocks + b;
    const bool valid = blk < I.nblk;
    int by = 0, bx = 0;
    if (valid) block_row_col(I.div_magic, I.nbx, blk, by, bx);
    uint4 raw[IO::kVec];
    if (valid) {
      IO::load(static_cast<const char*>(I.src) + (int64_t(by) * 16 + l) * I.src_pitch +
                   int64_t(bx) * 16 * int64_t(sizeof(Smp)),
               raw);
    } else {
#pragma unroll
      for (int q = 0; q < IO::kVec; ++q) raw[q] = make_uint4(0, 0, 0, 0);
    }
    int xs[16];
    IO::unpack(raw, xs);
    const bool quant = (I.flags & kQuantFlag) != 0;
    const int peak = (1 << (I.flags & 0xff)) - 1;

    // ---------------- one 16x16 block with T ----------------
    int p16[16];
    {
      int x[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = xs[j];
      __syncwarp();
      fwd16(x);
#pragma unroll
      for (int j = 0; j < 16; ++j) S[l][j] = x[j];
      __syncwarp();
      int lev[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) lev[u] = S[u][l];
      fwd16(lev);
      const int v = l;
      const int hcol = I.colh[v];
      if (quant) {
        const int ev = scale_class(v);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float ff = I.f[scale_class(u) + ev];
          lev[u] = u < hcol ? int(roundf(__fmul_rn(__int2float_rn(lev[u]), ff))) : 0;
        }
        inverse_to_row<true>(S, l, lev, I, p16);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) lev[u] = u < hcol ? lev[u] : 0;
        inverse_to_row<false>(S, l, lev, I, p16);
      }
    }

    // ---------------- four 8x8 blocks with T8 ----------------
    int p8[16];
    {
      int xa[8], xb[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        xa[j] = xs[j];
        xb[j] = xs[8 + j];
      }
      fwd8(xa);
      fwd8(xb);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        S8[l][j] = xa[j];
        S8[l][8 + j] = xb[j];
      }
      __syncwarp();
      // thread l: column v = l of the upper (rows 0..7) and lower (8..15) blocks
      const int v = l;
      const int vv = v & 7;
      int ca[8], cb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        ca[u] = S8[u][v];
        cb[u] = S8[8 + u][v];
      }
      fwd8(ca);
      fwd8(cb);
      const int h8 = M.colh8[vv];
      const int cv = c8(vv);
      if (quant) {
        float wa[8], wb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int kk = c8(u) + cv;
          const float ff = M.f8[kk], gg = M.g8[kk];
          const int la = u < h8 ? int(roundf(__fmul_rn(__int2float_rn(ca[u]), ff))) : 0;
          const int lb = u < h8 ? int(roundf(__fmul_rn(__int2float_rn(cb[u]), ff))) : 0;
          wa[u] = __fmul_rn(__int2float_rn(la), gg);
          wb[u] = __fmul_rn(__int2float_rn(lb), gg);
        }
        inv8(wa);
        inv8(wb);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          S8[u][v] = __float_as_int(wa[u]);
          S8[8 + u][v] = __float_as_int(wb[u]);
        }
        __syncwarp();
        float za[8], zb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          za[j] = __int_as_float(S8[l][j]);
          zb[j] = __int_as_float(S8[l][8 + j]);
        }
        inv8(za);
        inv8(zb);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          p8[j] = int(fminf(fmaxf(roundf(za[j]), 0.f), float(peak)));
          p8[8 + j] = int(fminf(fmaxf(roundf(zb[j]), 0.f), float(peak)));
        }
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int sh = c8(u) + cv;  // D8_u D8_v = 2^(c(u) + c(v))
          ca[u] = u < h8 ? ca[u] * (1 << sh) : 0;
          cb[u] = u < h8 ? cb[u] * (1 << sh) : 0;
        }
        inv8(ca);
        inv8(cb);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          S8[u][v] = ca[u];
          S8[8 + u][v] = cb[u];
        }
        __syncwarp();
        int za[8], zb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          za[j] = S8[l][j];
          zb[j] = S8[l][8 + j];
        }
        inv8(za);  // 64 X_tilde
        inv8(zb);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          p8[j] = min(max(round_div64(za[j]), 0), peak);
          p8[8 + j] = min(max(round_div64(zb[j]), 0), peak);
        }
      }
    }

    // ---------------- choose the tiling of the region ----------------
    unsigned e16 = 0, e8 = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      e16 += unsigned((xs[j] - p16[j]) * (xs[j] - p16[j]));
      e8 += unsigned((xs[j] - p8[j]) * (xs[j] - p8[j]));
    }
    // region totals over the 16 rows (lanes of one half-warp; 16 x 16 x 4095^2 < 2^32)
    unsigned t16 = e16, t8 = e8;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      t16 += __shfl_xor_sync(0xffffffffu, t16, o, 16);
      t8 += __shfl_xor_sync(0xffffffffu, t8, o, 16);
    }
    const bool split = M.mode == 2 || (M.mode == 0 && t8 < t16);
    if (valid) {
      if (I.dst != nullptr) {
        char* row = static_cast<char*>(I.dst) + (int64_t(by) * 16 + l) * I.dst_pitch +
                    int64_t(bx) * 16 * int64_t(sizeof(Smp));
        IO::store(row, split ? p8 : p16);
      }
      if (P.split && l == 0) P.split[I.blk0 + blk] = split ? 1 : 0;
      acc += split ? e8 : e16;
    }
  }
  if (P.sse) flush_sse_rows(P.sse, P.img[acc_img].p.out_index, acc);
}

template <typename Smp>
tx16_status launch_mixed(const MixedParam* imgs, int n, unsigned long long* sse, uint8_t* split,
                         cudaStream_t stream) {
  MixedBatch<kMixMaxImg> P;
  P.nimg = n;
  P.sse = sse;
  P.split = split;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].p.tile0 = tiles;
    tiles += (imgs[i].p.nblk + kTileBlocks - 1) / kTileBlocks;
  }
  P.ntiles = tiles;
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, mixed_kernel<Smp, kMixMaxImg>, kThreads, 0) !=
            cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min(tiles, occ * device_sm_count()));
  mixed_kernel<Smp, kMixMaxImg><<<grid, kThreads, 0, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

// Column heights of the first r cells of the 8x8 zig-zag scan (JPEG order).
void zonal_column_heights8(int r, uint8_t colh[8]) {
  int rank[8][8];
  int k = 0;
  for (int d = 0; d <= 14; ++d) {
    const int ulo = d < 8 ? 0 : d - 7;
    const int uhi = d < 8 ? d : 7;
    if (d & 1) {
      for (int u = ulo; u <= uhi; ++u) rank[u][d - u] = k++;
    } else {
      for (int u = uhi; u >= ulo; --u) rank[u][d - u] = k++;
    }
  }
  for (int v = 0; v < 8; ++v) {
    int h = 0;
    for (int u = 0; u < 8; ++u) h += rank[u][v] < r ? 1 : 0;
    colh[v] = uint8_t(h);
  }
}

}  // namespace
}  // namespace tx16

using namespace tx16;

extern "C" tx16_status tx16_codec_mixed(const tx16_image* in, const tx16_image* out, int32_t n,
                                        const tx16_mixed_qparams* qp, uint8_t* split, uint64_t* sse,
                                        void* stream) {
  TX16_TRACE("tx16_codec_mixed");
  if (n < 0 || (n > 0 && (in == nullptr || qp == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(sse) & 7u) != 0) return TX16_EINVAL;
  std::vector<MixedParam> M(n);
  int64_t blk0 = 0;
  for (int i = 0; i < n; ++i) {
    const tx16_mixed_qparams& m = qp[i];
    if (!valid_image(in[i])) return TX16_EINVAL;
    if (out != nullptr && (!valid_image(out[i]) || out[i].width != in[i].width || out[i].height != in[i].height ||
                           out[i].bits != in[i].bits))
      return TX16_EINVAL;
    if (!std::isfinite(m.q) || m.r16 < 1 || m.r16 > 256 || m.r8 < 1 || m.r8 > 64 || m.mode < 0 || m.mode > 2)
      return TX16_EINVAL;
    const tx16_qparams q16{m.q, m.r16};
    M[i].p = make_param(in[i], out ? &out[i] : nullptr, q16, blk0);
    M[i].p.out_index = i;
    blk0 += M[i].p.nblk;
    const double r2 = std::sqrt(2.0);
    for (int k = 0; k < 5; ++k) {
      const double ss = std::ldexp(1.0, -3 + k / 2) * ((k & 1) ? r2 : 1.0);  // 2^(-3 + k/2)
      M[i].f8[k] = m.q > 0.f ? float(ss / double(m.q)) : 0.f;
      M[i].g8[k] = m.q > 0.f ? float(double(m.q) * ss) : 0.f;
    }
    zonal_column_heights8(m.r8, M[i].colh8);
    M[i].mode = m.mode;
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sse != nullptr && cudaMemsetAsync(sse, 0, sizeof(uint64_t) * size_t(n), st) != cudaSuccess) return TX16_ECUDA;
  unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sse);
  // the one-region-per-thread kernel by class pair; the rest on the kernel
  // above, by runs of equal sample size
  std::vector<MixedParam> fast[kMixBtPairs], rest;
  for (int i = 0; i < n; ++i) {
    const int pair = mixed_bt_pair(M[i]);
    (pair >= 0 ? fast[pair] : rest).push_back(M[i]);
  }
  for (int c = 0; c < kMixBtPairs; ++c)
    for (size_t s = 0; s < fast[c].size(); s += kMixMaxImg) {
      const int m = int(std::min<size_t>(kMixMaxImg, fast[c].size() - s));
      const tx16_status r = launch_mixed_bt(c, fast[c].data() + s, m, s64, split, st);
      if (r != TX16_OK) return r;
    }
  const int nr = int(rest.size());
  int s = 0;
  while (s < nr) {
    const bool u8 = (rest[s].p.flags & 0xff) == 8;
    int e = s + 1;
    while (e < nr && e - s < kMixMaxImg && ((rest[e].p.flags & 0xff) == 8) == u8) ++e;
    const tx16_status r = u8 ? launch_mixed<uint8_t>(rest.data() + s, e - s, s64, split, st)
                             : launch_mixed<uint16_t>(rest.data() + s, e - s, s64, split, st);
    if (r != TX16_OK) return r;
    s = e;
  }
  return TX16_OK;
}
