// Images of any size (tx16_codec_any_size).  The paper's images split
// exactly into 16x16 blocks (Sec. 3.1); for other sizes the last row and the
// last column are repeated out to the next multiple of 16 (edge replication),
// the padded blocks are coded as usual, and only the image's own pixels are
// written and counted in the squared error.
//
// Each image is split on the host.  Where the one-block-per-thread kernel
// takes the image's samples and zone, its columns of whole blocks are coded
// over the full height by that kernel, which repeats the last row into a
// partial last block row in its loads and writes and counts only the image's
// rows.  Otherwise its interior of whole blocks goes to the ordinary codec
// kernels (a fused kernel where the samples and the step suit it, the general
// kernel otherwise) and the last, partial block row (interior width) to the
// strip kernel below.  The last, partial block column (full height) always
// goes to the strip kernel, which does the replication in its loads: a row
// below the image reads the last row instead, and samples right of the image
// take the value of the last column.  All launches add into the image's SSE
// slot.
//
// The strip kernel has the general kernel's mapping (16 threads per block,
// int32 forward, binary32 or exact inverse).  Colour images are coded plane
// by plane, one descriptor per plane (Sec. 3.1 codes each channel apart).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "tx16_block.cuh"
#include "tx16_internal.h"
#include "tx16_net.cuh"

namespace tx16 {
ImgParam make_param(const tx16_image& in, const tx16_image* out, const tx16_qparams& qp, int64_t blk0);
bool valid_qparams(const tx16_qparams& qp);

namespace {

struct AnyParam {
  ImgParam p;  // over the strip's padded block grid; p.out_index = SSE slot
  int32_t w, h;
};

template <int MAXI>
struct AnyBatch {
  int32_t nimg, ntiles;
  unsigned long long* sse;
  AnyParam img[MAXI];
};
constexpr int kAnyMaxImg = 240;
static_assert(sizeof(AnyBatch<kAnyMaxImg>) < 32000, "kernel parameters too large");

// 16 samples from p, of which the first wv lie inside the image.  The row's
// pitch is a multiple of 16 bytes and at least width samples, so the 16-byte
// vector holding sample wv - 1 lies inside the row; the second half of a
// 16-bit row is read only when it holds image samples.
template <typename Smp>
__device__ __forceinline__ void load_any(const void* p, int wv, uint4 (&w)[RowIO<Smp>::kVec]) {
  w[0] = __ldcs(reinterpret_cast<const uint4*>(p));
  if (RowIO<Smp>::kVec == 2)
    w[RowIO<Smp>::kVec - 1] = wv > 8 ? __ldcs(reinterpret_cast<const uint4*>(p) + 1) : make_uint4(0, 0, 0, 0);
}

template <typename Smp>
__device__ __forceinline__ void store_partial(void* row, const int (&p)[16], int n) {
  Smp* q = static_cast<Smp*>(row);
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < n) q[j] = Smp(p[j]);
}

template <typename Smp, int MAXI>
__global__ void __launch_bounds__(kThreads) any_size_kernel(const __grid_constant__ AnyBatch<MAXI> P) {
  __shared__ int sm[kTileBlocks][16][17];
  const int l = threadIdx.x & 15;
  const int b = threadIdx.x >> 4;
  int(*S)[17] = sm[b];
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
    const AnyParam& A = P.img[k];
    const ImgParam& I = A.p;
    const int blk = (t - I.tile0) * kTileBlocks + b;
    const bool valid = blk < I.nblk;
    int by = 0, bx = 0;
    if (valid) block_row_col(I.div_magic, I.nbx, blk, by, bx);
    const int y = by * 16 + l;                 // image row of this thread's block row
    const int ysrc = min(y, A.h - 1);          // rows below the image repeat the last row
    const int x0 = bx * 16;
    const int wv = min(16, A.w - x0);          // columns of this block inside the image (>= 1)
    uint4 raw[IO::kVec];
    if (valid) {
      load_any<Smp>(static_cast<const char*>(I.src) + int64_t(ysrc) * I.src_pitch + int64_t(x0) * int64_t(sizeof(Smp)),
                    wv, raw);
    } else {
#pragma unroll
      for (int q = 0; q < IO::kVec; ++q) raw[q] = make_uint4(0, 0, 0, 0);
    }
    int x[16];
    IO::unpack(raw, x);
    int last = x[0];
#pragma unroll
    for (int j = 0; j < 16; ++j) {  // columns right of the image repeat the last column
      if (j < wv) last = x[j];
      else x[j] = last;
    }
    int xs[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) xs[j] = x[j];
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
    const bool quant = (I.flags & kQuantFlag) != 0;
    if (quant) {
      const int ev = scale_class(v);
      const float f0 = I.f[ev], f1 = I.f[ev + 1], f2 = I.f[ev + 2];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int eu = scale_class(u);
        const float ff = eu == 0 ? f0 : (eu == 1 ? f1 : f2);
        lev[u] = u < hcol ? int(roundf(__fmul_rn(__int2float_rn(lev[u]), ff))) : 0;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 16; ++u) lev[u] = u < hcol ? lev[u] : 0;
    }
    int p[16];
    if (quant) inverse_to_row<true>(S, l, lev, I, p);
    else inverse_to_row<false>(S, l, lev, I, p);
    if (valid && y < A.h) {
      if (I.dst != nullptr) {
        char* row = static_cast<char*>(I.dst) + int64_t(y) * I.dst_pitch + int64_t(x0) * int64_t(sizeof(Smp));
        if (wv == 16) IO::store(row, p);
        else store_partial<Smp>(row, p, wv);
      }
      unsigned s = 0;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < wv) s += unsigned((xs[j] - p[j]) * (xs[j] - p[j]));
      acc += s;
    }
  }
  if (P.sse) flush_sse_rows(P.sse, P.img[acc_img].p.out_index, acc);
}

template <typename Smp>
tx16_status launch_any(const AnyParam* imgs, int n, unsigned long long* sse, cudaStream_t stream) {
  AnyBatch<kAnyMaxImg> P;
  P.nimg = n;
  P.sse = sse;
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, any_size_kernel<Smp, kAnyMaxImg>, kThreads, 0) !=
            cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  const int grid = std::max(1, std::min(tiles, occ * device_sm_count()));
  any_size_kernel<Smp, kAnyMaxImg><<<grid, kThreads, 0, stream>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

// An image of any size: the rules of valid_image() except that width and
// height need not be multiples of 16.  On success pad describes the padded
// block grid (width and height rounded up to 16, same data and pitch).
bool padded_descriptor(const tx16_image& im, tx16_image& pad) {
  if (im.data == nullptr || (reinterpret_cast<uintptr_t>(im.data) & 15u) != 0) return false;
  if (im.bits < 8 || im.bits > 12) return false;
  if (im.width <= 0 || im.height <= 0) return false;
  if (im.pitch_bytes <= 0 || (im.pitch_bytes % 16) != 0) return false;
  if (im.pitch_bytes < int64_t(im.width) * sample_bytes(im.bits)) return false;
  pad = im;
  pad.width = int32_t((int64_t(im.width) + 15) / 16 * 16);
  pad.height = int32_t((int64_t(im.height) + 15) / 16 * 16);
  if (pad.width <= 0 || pad.height <= 0) return false;
  return int64_t(pad.width / 16) * int64_t(pad.height / 16) <= (int64_t(1) << 30);
}

}  // namespace
}  // namespace tx16

using namespace tx16;

extern "C" tx16_status tx16_codec_any_size(const tx16_image* in, const tx16_image* out, int32_t n,
                                           const tx16_qparams* qp, uint64_t* sse, void* stream) {
  TX16_TRACE("tx16_codec_any_size");
  if (n < 0 || (n > 0 && (in == nullptr || qp == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(sse) & 7u) != 0) return TX16_EINVAL;
  // interior of whole blocks (width and height rounded down to 16) per image,
  // or nblk = 0 when there is none; edge strips as AnyParam
  std::vector<ImgParam> inner(n);
  std::vector<ImgParam> ragged;  // whole images of ragged height for the one-block-per-thread kernel
  std::vector<AnyParam> strips;
  strips.reserve(2 * size_t(n));
  for (int i = 0; i < n; ++i) {
    tx16_image pin, pout;
    if (!padded_descriptor(in[i], pin) || !valid_qparams(qp[i])) return TX16_EINVAL;
    if (out != nullptr && (!padded_descriptor(out[i], pout) || out[i].width != in[i].width ||
                           out[i].height != in[i].height || out[i].bits != in[i].bits))
      return TX16_EINVAL;
    const int esz = sample_bytes(in[i].bits);
    const int W = in[i].width, H = in[i].height;
    const int W16 = W / 16 * 16, H16 = H / 16 * 16;
    // a sub-image of in[i] / out[i] at (x, y), w x h samples
    auto sub = [&](const tx16_image& im, int x, int y, int w, int h) {
      tx16_image r = im;
      r.data = static_cast<char*>(im.data) + int64_t(y) * im.pitch_bytes + int64_t(x) * esz;
      r.width = w;
      r.height = h;
      return r;
    };
    std::memset(&inner[i], 0, sizeof(ImgParam));
    bool whole_height = false;  // columns [0, W16) over the full height coded as one ragged image
    if (W16 > 0 && H16 < H) {
      const int Hp = (H + 15) / 16 * 16;
      tx16_image a = sub(in[i], 0, 0, W16, Hp), b;
      if (out != nullptr) b = sub(out[i], 0, 0, W16, Hp);
      ImgParam p = make_param(a, out ? &b : nullptr, qp[i], 0);
      if (fused_bt_ragged_supports(p)) {
        p.flags |= (Hp - H) << kBtMissingShift;
        p.out_index = i;
        ragged.push_back(p);
        whole_height = true;
      }
    }
    if (W16 > 0 && H16 > 0 && !whole_height) {
      const tx16_image a = sub(in[i], 0, 0, W16, H16);
      tx16_image b;
      if (out != nullptr) b = sub(out[i], 0, 0, W16, H16);
      inner[i] = make_param(a, out ? &b : nullptr, qp[i], 0);
    }
    auto add_strip = [&](int x, int y, int w, int h) {
      tx16_image a = sub(in[i], x, y, w, h), pa, pb;
      padded_descriptor(a, pa);  // x * esz is a multiple of 16: alignment and pitch rules carry over
      tx16_image b;
      if (out != nullptr) {
        b = sub(out[i], x, y, w, h);
        padded_descriptor(b, pb);
      }
      AnyParam A;
      A.p = make_param(pa, out ? &pb : nullptr, qp[i], 0);
      A.p.out_index = i;
      A.w = w;
      A.h = h;
      strips.push_back(A);
    };
    if (W16 < W) add_strip(W16, 0, W - W16, H);   // last block column, full height
    if (H16 < H && W16 > 0 && !whole_height) add_strip(0, H16, W16, H - H16);  // last block row, interior width
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sse != nullptr && cudaMemsetAsync(sse, 0, sizeof(uint64_t) * size_t(n), st) != cudaSuccess) return TX16_ECUDA;
  unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sse);
  // interiors: runs of consecutive images that have one, by kernel
  int s = 0;
  while (s < n) {
    if (inner[s].nblk == 0) {
      ++s;
      continue;
    }
    int e = s + 1;
    while (e < n && inner[e].nblk > 0) ++e;
    const tx16_status r = launch_codec_runs(inner.data() + s, e - s, s64 ? s64 + s : nullptr, nullptr, st);
    if (r != TX16_OK) return r;
    s = e;
  }
  // whole images of ragged height
  if (!ragged.empty()) {
    const tx16_status r = launch_fused_bt_ragged(ragged.data(), int(ragged.size()), s64, st);
    if (r != TX16_OK) return r;
  }
  // edge strips: runs of equal sample size, at most kAnyMaxImg per launch
  const int m = int(strips.size());
  s = 0;
  while (s < m) {
    const bool u8 = (strips[s].p.flags & 0xff) == 8;
    int e = s + 1;
    while (e < m && e - s < kAnyMaxImg && ((strips[e].p.flags & 0xff) == 8) == u8) ++e;
    const tx16_status r = u8 ? launch_any<uint8_t>(strips.data() + s, e - s, s64, st)
                             : launch_any<uint16_t>(strips.data() + s, e - s, s64, st);
    if (r != TX16_OK) return r;
    s = e;
  }
  return TX16_OK;
}
