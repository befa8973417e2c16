// Block kernels of libtx16: forward transform, fused codec, inverse, and the
// squared-error reduction of the unfused form.
//
// Work decomposition (Sec. 3.1 splits every image into disjoint 16x16 blocks):
//   * a tile is 16 consecutive blocks of one image in raster block order;
//   * a CTA of 256 threads works on one tile at a time: half-warp b owns block
//     b of the tile and its thread l owns row l of that block;
//   * each CTA walks a contiguous range of tiles (grid sized to fill the SMs),
//     so per-image squared errors stay in registers until the image changes.
//
// Per block: the row pass (T on each row) runs on the row held by each thread;
// the row/column exchange goes through 1 KB of shared memory (16 x 17 words,
// conflict-free both ways); the column pass leaves column v of Y = T X T^t in
// thread v; quantisation and the inverse column pass need no exchange; one more
// exchange returns rows for the inverse row pass, rounding and the store.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>

#include "tx16_block.cuh"
#include "tx16_internal.h"
#include "tx16_net.cuh"

namespace tx16 {

template <typename Smp, int MAXI, int OP>
__global__ void __launch_bounds__(kThreads) block_kernel(const __grid_constant__ BatchParams<MAXI> P) {
  __shared__ int sm[kTileBlocks][16][17];
  const int l = threadIdx.x & 15;
  const int b = threadIdx.x >> 4;
  int(*S)[17] = sm[b];
  using IO = RowIO<Smp>;

  const int per = (P.ntiles + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per;
  const int t1 = min(t0 + per, P.ntiles);
  if (t0 >= t1) return;  // uniform over the CTA

  int k = 0;  // image of tile t0: the last one with tile0 <= t0
  {
    int hi = P.nimg - 1;
    while (k < hi) {
      const int mid = (k + hi + 1) >> 1;
      if (P.img[mid].tile0 <= t0) k = mid; else hi = mid - 1;
    }
  }
  unsigned long long acc = 0;
  int acc_img = k;

  for (int t = t0; t < t1; ++t) {
    while (k + 1 < P.nimg && P.img[k + 1].tile0 <= t) ++k;  // uniform
    if (OP == kOpCodec || OP == kOpSse) {
      if (k != acc_img) {
        if (P.sse) flush_sse_rows(P.sse, acc_img, acc);
        acc = 0;
        acc_img = k;
      }
    }
    const ImgParam& I = P.img[k];
    const int blk = (t - I.tile0) * kTileBlocks + b;
    const bool valid = blk < I.nblk;
    int by = 0, bx = 0;
    if (valid) block_row_col(I.div_magic, I.nbx, blk, by, bx);
    const int64_t row = int64_t(by) * 16 + l;
    const int64_t col_bytes = int64_t(bx) * 16 * int64_t(sizeof(Smp));

    __syncwarp();
    if (OP == kOpSse) {
      uint4 ra[IO::kVec], rb[IO::kVec];
      if (valid) {
        IO::load(static_cast<const char*>(I.src) + row * I.src_pitch + col_bytes, ra);
        IO::load(static_cast<const char*>(I.dst) + row * I.dst_pitch + col_bytes, rb);
        int xa[16], xb[16];
        IO::unpack(ra, xa);
        IO::unpack(rb, xb);
        unsigned s = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) s += unsigned((xa[j] - xb[j]) * (xa[j] - xb[j]));
        acc += s;
      }
      continue;
    }

    int lev[16];  // column v = l of Y (forward/codec) or of the levels (inverse)
    uint4 raw[IO::kVec];
    if (OP == kOpForward || OP == kOpCodec) {
      if (valid) {
        IO::load(static_cast<const char*>(I.src) + row * I.src_pitch + col_bytes, raw);
      } else {
#pragma unroll
        for (int q = 0; q < IO::kVec; ++q) raw[q] = make_uint4(0, 0, 0, 0);
      }
      int x[16];
      IO::unpack(raw, x);
      fwd16(x);  // row pass: x[k] = (X T^t)[l][k]
#pragma unroll
      for (int j = 0; j < 16; ++j) S[l][j] = x[j];
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 16; ++u) lev[u] = S[u][l];
      fwd16(lev);  // column pass: lev[u] = Y[u][v], v = l
      if (OP == kOpForward) {
        if (valid) {
          int* out = P.coeffs + (I.blk0 + blk) * 256 + l;
#pragma unroll
          for (int u = 0; u < 16; ++u) __stcs(out + 16 * u, lev[u]);
        }
        continue;
      }
    }

    const int v = l;
    const int h = I.colh[v];
    const bool quant = (I.flags & kQuantFlag) != 0;
    if (OP == kOpInverse) {
      const int* in = P.coeffs + (I.blk0 + blk) * 256 + v;
#pragma unroll
      for (int u = 0; u < 16; ++u) lev[u] = (valid && u < h) ? __ldcs(in + 16 * u) : 0;
    } else {
      // zonal mask and quantiser (Sec. 3.1; S merged into the quantiser)
      if (quant) {
        const int ev = scale_class(v);
        const float f0 = I.f[ev], f1 = I.f[ev + 1], f2 = I.f[ev + 2];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int eu = scale_class(u);
          const float ff = eu == 0 ? f0 : (eu == 1 ? f1 : f2);
          lev[u] = u < h ? int(roundf(__fmul_rn(__int2float_rn(lev[u]), ff))) : 0;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) lev[u] = u < h ? lev[u] : 0;
      }
      if (P.coeffs != nullptr && valid) {
        int* out = P.coeffs + (I.blk0 + blk) * 256 + v;
#pragma unroll
        for (int u = 0; u < 16; ++u) __stcs(out + 16 * u, lev[u]);
      }
    }

    int p[16];
    if (quant) inverse_to_row<true>(S, l, lev, I, p);
    else inverse_to_row<false>(S, l, lev, I, p);

    if (valid && I.dst != nullptr)
      IO::store(static_cast<char*>(I.dst) + row * I.dst_pitch + col_bytes, p);
    if (OP == kOpCodec && valid) {
      int x[16];
      IO::unpack(raw, x);
      unsigned s = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) s += unsigned((x[j] - p[j]) * (x[j] - p[j]));
      acc += s;
    }
  }
  if ((OP == kOpCodec || OP == kOpSse) && P.sse) flush_sse_rows(P.sse, acc_img, acc);
}

// Elementwise quantiser of the unfused form: 4 coefficients per thread.
struct QuantParams {
  float f[5];
  uint8_t colh[16];
  int32_t quant;
};

__global__ void __launch_bounds__(256) quantise_kernel(const int4* __restrict__ in, int4* __restrict__ out,
                                                       int64_t n4, const QuantParams Q) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n4;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int e = int(i & 63) * 4;  // element index inside the block
    const int u = e >> 4, v0 = e & 15;
    const int4 y = __ldcs(in + i);
    int yy[4] = {y.x, y.y, y.z, y.w};
    const int eu = scale_class(u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int v = v0 + j;
      const bool keep = u < Q.colh[v];
      if (Q.quant) {
        const float ff = Q.f[eu + scale_class(v)];
        yy[j] = keep ? int(roundf(__fmul_rn(__int2float_rn(yy[j]), ff))) : 0;
      } else {
        yy[j] = keep ? yy[j] : 0;
      }
    }
    __stcs(out + i, make_int4(yy[0], yy[1], yy[2], yy[3]));
  }
}

// ---------------------------------------------------------------------------
// Launch
// ---------------------------------------------------------------------------
int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (cached[dev] == 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = sms > 0 ? sms : 1;
  }
  return cached[dev];
}

template <typename Smp, int MAXI, int OP>
static tx16_status launch_one(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* coeffs,
                              cudaStream_t stream) {
  BatchParams<MAXI> P;
  P.nimg = n;
  P.sse = sse;
  P.coeffs = coeffs;
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].tile0 = tiles;
    tiles += (imgs[i].nblk + kTileBlocks - 1) / kTileBlocks;
  }
  P.ntiles = tiles;
  static std::atomic<int> occ{0};  // resident CTAs per SM for this instance (same on every GB300)
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, block_kernel<Smp, MAXI, OP>, kThreads, 0) !=
            cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min(tiles, occ * device_sm_count()));
  block_kernel<Smp, MAXI, OP><<<grid, kThreads, 0, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

template <typename Smp, int OP>
static tx16_status launch_sized(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* coeffs,
                                cudaStream_t stream) {
  if (n == 1) return launch_one<Smp, 1, OP>(imgs, n, sse, coeffs, stream);
  if (n <= 32) return launch_one<Smp, 32, OP>(imgs, n, sse, coeffs, stream);
  return launch_one<Smp, kMaxImg, OP>(imgs, n, sse, coeffs, stream);
}

template <int OP>
static tx16_status launch_op(int sbytes, const ImgParam* imgs, int n, unsigned long long* sse,
                             int32_t* coeffs, cudaStream_t stream) {
  return sbytes == 1 ? launch_sized<uint8_t, OP>(imgs, n, sse, coeffs, stream)
                     : launch_sized<uint16_t, OP>(imgs, n, sse, coeffs, stream);
}

tx16_status launch_blocks(Op op, int sbytes, ImgParam* imgs, int n, unsigned long long* sse,
                          int32_t* coeffs, cudaStream_t stream) {
  for (int s = 0; s < n; s += kMaxImg) {
    const int m = std::min(kMaxImg, n - s);
    unsigned long long* sse_s = sse ? sse + s : nullptr;
    tx16_status st;
    switch (op) {
      case kOpForward: st = launch_op<kOpForward>(sbytes, imgs + s, m, sse_s, coeffs, stream); break;
      case kOpCodec: st = launch_op<kOpCodec>(sbytes, imgs + s, m, sse_s, coeffs, stream); break;
      case kOpInverse: st = launch_op<kOpInverse>(sbytes, imgs + s, m, sse_s, coeffs, stream); break;
      default: st = launch_op<kOpSse>(sbytes, imgs + s, m, sse_s, coeffs, stream); break;
    }
    if (st != TX16_OK) return st;
  }
  return TX16_OK;
}

tx16_status launch_quantise(const int32_t* coeffs, int64_t nblk, const ImgParam& qp, int32_t* levels,
                            cudaStream_t stream) {
  QuantParams Q;
  for (int k = 0; k < 5; ++k) Q.f[k] = qp.f[k];
  for (int v = 0; v < 16; ++v) Q.colh[v] = qp.colh[v];
  Q.quant = (qp.flags & kQuantFlag) ? 1 : 0;
  const int64_t n4 = nblk * 64;
  const int64_t want = (n4 + 255) / 256;
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 8)));
  quantise_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const int4*>(coeffs),
                                            reinterpret_cast<int4*>(levels), n4, Q);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

}  // namespace tx16
