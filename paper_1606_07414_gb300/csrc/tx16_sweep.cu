// Zonal sweep (tx16_zonal_sweep): the paper's image experiment for several r
// at once (Sec. 3.1 zonal coding; Fig. 2 plots PSNR per additive cost against
// r).  Each block is transformed forward once, exactly; then, for every r of
// the list, the coefficients outside Z_r are zeroed and the block is
// reconstructed exactly (256 X = T^t (D' Y D') T over the kept cells, no
// quantiser), rounded, clipped and compared with the input.  One launch gives
// the squared error of every (image, r) pair.
//
// Mapping: 16 threads per block (thread l: row l, then column v = l), 16
// blocks per CTA, int32 networks (tx16_net.cuh), row/column exchange through
// a 16 x 17-word shared buffer per block; each r's squared error is summed
// over the warp by shuffles into a per-warp shared-memory slot, flushed with
// one atomic per warp and r when the image changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "tx16_internal.h"
#include "tx16_net.cuh"

namespace tx16 {

constexpr int kSweepMaxR = 16;

struct SweepImg {
  const void* src;
  int64_t pitch;
  int32_t nbx, nblk, tile0, bits;
  uint32_t div_magic;
};

template <int MAXI>
struct SweepParams {
  int32_t nimg, ntiles, nr;
  unsigned long long* sse;  // [image][r]
  uint8_t colh[kSweepMaxR][16];
  SweepImg img[MAXI];
};
constexpr int kSweepMaxImg = 200;
static_assert(sizeof(SweepParams<kSweepMaxImg>) < 32000, "kernel parameters too large");

namespace {

template <typename Smp>
__device__ __forceinline__ void load_row(const void* p, int (&x)[16]) {
  if (sizeof(Smp) == 1) {
    const uint4 w = __ldcs(reinterpret_cast<const uint4*>(p));
    const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (u[k >> 2] >> (8 * (k & 3))) & 0xffu;
  } else {
    const uint4 w0 = __ldcs(reinterpret_cast<const uint4*>(p));
    const uint4 w1 = __ldcs(reinterpret_cast<const uint4*>(p) + 1);
    const unsigned u[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (u[k >> 1] >> (16 * (k & 1))) & 0xffffu;
  }
}

template <typename Smp, int MAXI>
__global__ void __launch_bounds__(256) sweep_kernel(const __grid_constant__ SweepParams<MAXI> P) {
  __shared__ int sm[16][16][17];
  // per warp and r: squared error of the current image (lane 0 of the warp
  // adds the warp's sum after each block pair; flushed on an image change)
  __shared__ unsigned long long wacc[8][kSweepMaxR];
  const int l = threadIdx.x & 15;
  const int b = threadIdx.x >> 4;
  const int wib = threadIdx.x >> 5;
  int(*Sx)[17] = sm[b];
  const int per = (P.ntiles + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per;
  const int t1 = min(t0 + per, P.ntiles);
  if (t0 >= t1) return;
  int k = 0;
  while (k + 1 < P.nimg && P.img[k + 1].tile0 <= t0) ++k;
  if ((threadIdx.x & 31) < kSweepMaxR) wacc[wib][threadIdx.x & 31] = 0;
  __syncwarp();
  int acc_img = k;
  const int ev = scale_class(l);

  auto flush = [&](int img) {  // lane i < nr flushes r number i of its warp
    __syncwarp();
    const int i = threadIdx.x & 31;
    if (i < P.nr) {
      const unsigned long long v = wacc[wib][i];
      if (v) atomicAdd(P.sse + int64_t(img) * P.nr + i, v);
      wacc[wib][i] = 0;
    }
    __syncwarp();
  };

  for (int t = t0; t < t1; ++t) {
    while (k + 1 < P.nimg && P.img[k + 1].tile0 <= t) ++k;  // uniform
    if (k != acc_img) {
      flush(acc_img);
      acc_img = k;
    }
    const SweepImg& I = P.img[k];
    const int blk = (t - I.tile0) * 16 + b;
    const bool valid = blk < I.nblk;
    int by = 0, bx = 0;
    if (valid) {
      by = int(__umulhi(unsigned(blk), I.div_magic));
      bx = blk - by * I.nbx;
      if (bx >= I.nbx) {
        ++by;
        bx -= I.nbx;
      }
    }
    int x0[16];
    if (valid) {
      load_row<Smp>(static_cast<const char*>(I.src) + (int64_t(by) * 16 + l) * I.pitch +
                        int64_t(bx) * 16 * int64_t(sizeof(Smp)),
                    x0);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) x0[j] = 0;
    }
    const int peak = (1 << I.bits) - 1;
    // forward, once: Y[:, v] in thread v
    int x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = x0[j];
    fwd16(x);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) Sx[l][j] = x[j];
    __syncwarp();
    int y[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) y[u] = Sx[u][l];
    fwd16(y);
    // D' Y D' for column v = l (exact; masked per r below)
#pragma unroll
    for (int u = 0; u < 16; ++u) y[u] *= (1 << (scale_class(u) + ev));
    for (int ri = 0; ri < P.nr; ++ri) {  // uniform loop over the r list
      const int h = P.colh[ri][l];
      int w[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) w[u] = u < h ? y[u] : 0;
      inv16(w);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 16; ++i) Sx[i][l] = w[i];
      __syncwarp();
      int z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = Sx[l][j];
      inv16(z);  // 256 X_tilde of row l
      unsigned s = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        // round half away from zero of n / 256, clipped: a negative n
        // clips to 0 whichever way it rounds, so floor((n + 128) / 256)
        // (arithmetic shift) serves for every n
        const int pv = min(max((z[j] + 128) >> 8, 0), peak);
        const int d = x0[j] - pv;
        s += unsigned(d * d);
      }
      if (!valid) s = 0;
      // the warp's sum for this r (two blocks, 32 rows), added by lane 0: in
      // 32 bits for 8-bit samples (at most 32 * 16 * 255^2 < 2^32), in 64
      // bits beyond
      unsigned long long v;
      if (sizeof(Smp) == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        v = s;
      } else {
        v = s;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      }
      if ((threadIdx.x & 31) == 0) wacc[wib][ri] += v;
    }
  }
  flush(acc_img);
}

template <typename Smp, int MAXI>
tx16_status launch_sweep(const SweepImg* imgs, int n, const uint8_t (*colh)[16], int nr, unsigned long long* sse,
                         cudaStream_t stream) {
  SweepParams<MAXI> P;
  P.nimg = n;
  P.nr = nr;
  P.sse = sse;
  for (int i = 0; i < nr; ++i)
    for (int v = 0; v < 16; ++v) P.colh[i][v] = colh[i][v];
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].tile0 = tiles;
    tiles += (imgs[i].nblk + 15) / 16;
  }
  P.ntiles = tiles;
  static std::atomic<int> occ{0};  // resident CTAs per SM, looked up once
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, sweep_kernel<Smp, MAXI>, 256, 0) != cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min(tiles, occ * device_sm_count()));
  sweep_kernel<Smp, MAXI><<<grid, 256, 0, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

}  // namespace
}  // namespace tx16

using namespace tx16;

extern "C" tx16_status tx16_zonal_sweep(const tx16_image* imgs, int32_t n, const int32_t* r_list, int32_t nr,
                                        uint64_t* sse, void* stream) {
  TX16_TRACE("tx16_zonal_sweep");
  if (n < 0 || nr < 1 || nr > kSweepMaxR || r_list == nullptr) return TX16_EINVAL;
  if (n > 0 && (imgs == nullptr || sse == nullptr)) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(sse) & 7u) != 0) return TX16_EINVAL;
  uint8_t colh[kSweepMaxR][16];
  for (int i = 0; i < nr; ++i) {
    if (r_list[i] < 1 || r_list[i] > 256) return TX16_EINVAL;
    zonal_column_heights(r_list[i], colh[i]);
  }
  std::vector<SweepImg> I(n);
  for (int i = 0; i < n; ++i) {
    if (!valid_image(imgs[i])) return TX16_EINVAL;
    I[i].src = imgs[i].data;
    I[i].pitch = imgs[i].pitch_bytes;
    I[i].nbx = imgs[i].width / 16;
    I[i].nblk = I[i].nbx * (imgs[i].height / 16);
    I[i].bits = imgs[i].bits;
    I[i].div_magic = I[i].nbx == 1 ? 0xFFFFFFFFu : uint32_t((uint64_t(1) << 32) / uint64_t(I[i].nbx));
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(sse, 0, sizeof(uint64_t) * size_t(n) * size_t(nr), st) != cudaSuccess) return TX16_ECUDA;
  unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sse);
  // runs of equal sample size, at most kSweepMaxImg images per launch
  int s = 0;
  while (s < n) {
    int e = s + 1;
    while (e < n && e - s < kSweepMaxImg && (imgs[e].bits == 8) == (imgs[s].bits == 8)) ++e;
    const tx16_status r = imgs[s].bits == 8
                              ? launch_sweep<uint8_t, kSweepMaxImg>(I.data() + s, e - s, colh, nr,
                                                                   s64 + int64_t(s) * nr, st)
                              : launch_sweep<uint16_t, kSweepMaxImg>(I.data() + s, e - s, colh, nr,
                                                                    s64 + int64_t(s) * nr, st);
    if (r != TX16_OK) return r;
    s = e;
  }
  return TX16_OK;
}
