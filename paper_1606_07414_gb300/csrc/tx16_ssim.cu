// SSIM (tx16_ssim): the paper's second quality measure (Sec. 3.1, Fig. 2(b),
// Fig. 3), with the window and constants of the article it cites (Wang, Bovik,
// Sheikh and Simoncelli, 2004): an 11 x 11 Gaussian window of standard
// deviation 1.5 normalised to unit sum, K1 = 0.01, K2 = 0.03, L = 2^bits - 1,
// statistics at every position where the window fits inside the image, and
// the mean of the local indices (MSSIM).
//
// The Gaussian window is the outer product of a normalised 1-D window g, so
// the five local moments (E x, E y, E x^2, E y^2, E xy) are two 11-tap passes:
// along rows into shared memory, then along columns in registers.  Samples are
// centred on 2^(bits-1) before squaring, which keeps E x^2 - (E x)^2 from
// cancelling more digits than it must; the luminance term adds the centre
// back.  All arithmetic is binary32; each CTA adds its partial mean into the
// image's binary64 result with one atomic.
//
// Mapping: a CTA owns a strip of 32 output columns and kSegRows output rows of
// one image and walks down it in chunks of 64 rows.  Per chunk: stage the new
// input rows (as centred floats; the words were fetched into registers during
// the previous chunk's column pass), the row pass for 64 (first chunk 74) rows
// of the five moment planes, then the column pass, 4 rows of a pair of
// columns per thread.  The last 10 rows of the moment planes move to the top
// for the next chunk.  The kernel is arithmetic-bound: 137.5 binary32
// operations per output (row pass 65.5: 10.5 products and 11 per moment with
// the window's symmetry; column pass 55; the index 17) against 2 sample
// reads; the column pass and the index run on packed pairs of columns
// (__ffma2_rn and friends: two operations per instruction).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "tx16_internal.h"

namespace tx16 {
namespace {

constexpr int kWin = 11;                   // window side
constexpr int kHalo = kWin - 1;            // 10
constexpr int kStripCols = 32;             // output columns per CTA
constexpr int kChunk = 64;                 // output rows per chunk
constexpr int kSegRows = 512;              // output rows per CTA
constexpr int kHRows = kChunk + kHalo;     // 74 moment rows held
constexpr int kInW = 44;                   // staged input columns (42 used, float4 reads)
constexpr int kSsimThreads = 256;
constexpr int kSsimMaxImg = 200;
constexpr size_t kSsimSmem = sizeof(float) * (2 * kHRows * kInW + 5 * kHRows * kStripCols);

struct SsimImg {
  const void* a;
  const void* b;
  int64_t pa, pb;        // pitches in bytes
  int64_t map_off;       // first element of this image's map
  double inv_count;      // 1 / number of window positions
  int32_t w, h;          // image size
  int32_t mw, mh;        // map size: w - 10, h - 10
  int32_t nstrips, unit0;
  float centre, c1, c2;
};

template <int MAXI>
struct SsimParams {
  int32_t nimg, nunits;
  double* mssim;
  float* map;
  float g[kWin];  // normalised 1-D Gaussian, binary32
  SsimImg img[MAXI];
};
static_assert(sizeof(SsimParams<kSsimMaxImg>) < 32000, "kernel parameters too large");

// Input staging.  Samples travel as aligned 4-sample words (4 bytes for
// 8-bit planes, 8 bytes for 16-bit ones) and become centred floats through
// the exponent trick: 0x4B000000 | v is the float 2^23 + v, so subtracting
// 2^23 + centre gives v - centre exactly.
template <typename Smp>
struct Word;
template <>
struct Word<uint8_t> {
  using T = unsigned;
  __device__ static __forceinline__ T load(const void* p) { return __ldg(static_cast<const unsigned*>(p)); }
  __device__ static __forceinline__ float get(T w, int j, float bias) {
    return __int_as_float(int(__byte_perm(w, 0x4B000000u, 0x7440u | unsigned(j)))) - bias;
  }
};
template <>
struct Word<uint16_t> {
  using T = uint2;
  __device__ static __forceinline__ T load(const void* p) { return __ldg(static_cast<const uint2*>(p)); }
  __device__ static __forceinline__ float get(T w, int j, float bias) {
    const unsigned src = j < 2 ? w.x : w.y;
    const unsigned lo = unsigned(2 * (j & 1));
    return __int_as_float(int(__byte_perm(src, 0x4B000000u, 0x7400u | ((lo + 1) << 4) | lo))) - bias;
  }
};

constexpr int kWords = (kStripCols + kHalo + 3) / 4;   // 11 words of 4 samples per staged row
constexpr int kStageRows = kSsimThreads / kWords;      // 23 rows per staging pass
constexpr int kStagePasses = (kHRows + kStageRows - 1) / kStageRows;  // 4

template <typename Smp, bool MAP, int MAXI>
__global__ void __launch_bounds__(kSsimThreads, sizeof(Smp) == 1 ? 3 : 2) ssim_kernel(const __grid_constant__ SsimParams<MAXI> P) {
  extern __shared__ __align__(16) float sm[];
  float* in_a = sm;                          // [kHRows][kInW]
  float* in_b = in_a + kHRows * kInW;        // [kHRows][kInW]
  float* hm = in_b + kHRows * kInW;          // [5][kHRows][kStripCols]
  const int tid = threadIdx.x;
  using Wd = Word<Smp>;

  // unit -> image (largest k with unit0 <= unit)
  const int unit = blockIdx.x;
  int lo = 0, hi = P.nimg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.img[mid].unit0 <= unit) lo = mid;
    else hi = mid - 1;
  }
  const SsimImg& I = P.img[lo];
  const int u = unit - I.unit0;
  const int strip = u % I.nstrips;
  const int seg = u / I.nstrips;
  const int c0 = strip * kStripCols;
  const int r_begin = seg * kSegRows;
  const int r_end = min(r_begin + kSegRows, I.mh);
  const float bias = 8388608.f + I.centre;

  // staging slot of this thread: word sw of rows sr, sr + 23, ...; the word
  // is read at ws (clamped so that it holds sample w - 1 when it starts past
  // it) and samples past the image take sample w - 1
  const bool stager = tid < kStageRows * kWords;
  const int sr = tid / kWords;
  const int sw = tid - sr * kWords;
  const int xw = c0 + 4 * sw;
  const int ws = min(xw, (I.w - 1) & ~3);
  int sel[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) sel[j] = min(xw + j, I.w - 1) - ws;
  typename Wd::T ra[kStagePasses], rb[kStagePasses];
  auto fetch = [&](int y0, int nrows) {
#pragma unroll
    for (int k = 0; k < kStagePasses; ++k) {
      const int rr = sr + k * kStageRows;
      if (stager && rr < nrows) {
        const int y = min(y0 + rr, I.h - 1);
        ra[k] = Wd::load(static_cast<const char*>(I.a) + int64_t(y) * I.pa + int64_t(ws) * int64_t(sizeof(Smp)));
        rb[k] = Wd::load(static_cast<const char*>(I.b) + int64_t(y) * I.pb + int64_t(ws) * int64_t(sizeof(Smp)));
      }
    }
  };
  auto stage = [&](int nrows) {
#pragma unroll
    for (int k = 0; k < kStagePasses; ++k) {
      const int rr = sr + k * kStageRows;
      if (stager && rr < nrows) {
        float4 fa, fb;
        fa.x = Wd::get(ra[k], sel[0], bias); fa.y = Wd::get(ra[k], sel[1], bias);
        fa.z = Wd::get(ra[k], sel[2], bias); fa.w = Wd::get(ra[k], sel[3], bias);
        fb.x = Wd::get(rb[k], sel[0], bias); fb.y = Wd::get(rb[k], sel[1], bias);
        fb.z = Wd::get(rb[k], sel[2], bias); fb.w = Wd::get(rb[k], sel[3], bias);
        *reinterpret_cast<float4*>(in_a + rr * kInW + 4 * sw) = fa;
        *reinterpret_cast<float4*>(in_b + rr * kInW + 4 * sw) = fb;
      }
    }
  };

  fetch(r_begin, kHRows);
  float sum = 0.f;
  for (int r0 = r_begin; r0 < r_end; r0 += kChunk) {
    const bool first = r0 == r_begin;
    const int nrows = first ? kHRows : kChunk;     // moment rows to compute
    const int dst0 = first ? 0 : kHalo;            // where they go
    if (!first) {
      // keep the last 10 moment rows: rows 64..73 -> 0..9 (float4 moves)
      constexpr int kPer = kHalo * kStripCols / 4;  // float4 per plane
      for (int i = tid; i < 5 * kPer; i += kSsimThreads) {
        const int q = i / kPer;
        const int o = i - q * kPer;
        float4* base = reinterpret_cast<float4*>(hm + q * kHRows * kStripCols);
        base[o] = base[kChunk * kStripCols / 4 + o];
      }
    }
    stage(nrows);
    __syncthreads();
    // row pass: 4 adjacent columns of one row per task; the window is
    // symmetric, so each tap pair is added before its weight multiplies it
    for (int task = tid; task < nrows * (kStripCols / 4); task += kSsimThreads) {
      const int rr = task >> 3;
      const int cg = task & 7;
      float va[16], vb[16];
      const float4* pa4 = reinterpret_cast<const float4*>(in_a + rr * kInW + 4 * cg);
      const float4* pb4 = reinterpret_cast<const float4*>(in_b + rr * kInW + 4 * cg);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float4 x4 = pa4[m], y4 = pb4[m];
        va[4 * m] = x4.x; va[4 * m + 1] = x4.y; va[4 * m + 2] = x4.z; va[4 * m + 3] = x4.w;
        vb[4 * m] = y4.x; vb[4 * m + 1] = y4.y; vb[4 * m + 2] = y4.z; vb[4 * m + 3] = y4.w;
      }
      float4* o = reinterpret_cast<float4*>(hm + (dst0 + rr) * kStripCols + 4 * cg);
      constexpr int kPlane = kHRows * kStripCols / 4;  // float4 per plane
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        float v[14];
#pragma unroll
        for (int i = 0; i < 14; ++i)
          v[i] = q == 0 ? va[i] : q == 1 ? vb[i] : q == 2 ? va[i] * va[i] : q == 3 ? vb[i] * vb[i] : va[i] * vb[i];
        float h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float acc = P.g[kHalo / 2] * v[j + kHalo / 2];
#pragma unroll
          for (int k = kHalo / 2 - 1; k >= 0; --k) acc = fmaf(P.g[k], v[j + k] + v[j + kHalo - k], acc);
          h[j] = acc;
        }
        o[q * kPlane] = make_float4(h[0], h[1], h[2], h[3]);
      }
    }
    __syncthreads();
    // the next chunk's samples are fetched now and land behind the column pass
    if (r0 + kChunk < r_end) fetch(r0 + kChunk + kHalo, kChunk);
    // column pass: columns 2 cp and 2 cp + 1 as one packed pair (each lane
    // the same binary32 operations as a scalar pass), output rows
    // r0 + 4 rg .. r0 + 4 rg + 3
    {
      const int cp = tid & 15;
      const int rg = tid >> 4;
      float2 e[5][4];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        float2 v[4 + kHalo];
#pragma unroll
        for (int m = 0; m < 4 + kHalo; ++m)
          v[m] = *reinterpret_cast<const float2*>(hm + (q * kHRows + 4 * rg + m) * kStripCols + 2 * cp);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < kWin; ++k) acc = __ffma2_rn(make_float2(P.g[k], P.g[k]), v[i + k], acc);
          e[q][i] = acc;
        }
      }
      const int x = c0 + 2 * cp;
      const float2 centre = make_float2(I.centre, I.centre);
      const float2 c1 = make_float2(I.c1, I.c1), c2 = make_float2(I.c2, I.c2);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int y = r0 + 4 * rg + i;
        const float2 mxp = e[0][i], myp = e[1][i];
        const float2 nmx = make_float2(-mxp.x, -mxp.y), nmy = make_float2(-myp.x, -myp.y);
        const float2 sxx = __ffma2_rn(nmx, mxp, e[2][i]);
        const float2 syy = __ffma2_rn(nmy, myp, e[3][i]);
        const float2 sxy = __ffma2_rn(nmx, myp, e[4][i]);
        const float2 mx = __fadd2_rn(mxp, centre), my = __fadd2_rn(myp, centre);
        const float2 n1 = __ffma2_rn(__fadd2_rn(mx, mx), my, c1);  // mx + mx = 2 mx exactly
        const float2 d1 = __ffma2_rn(mx, mx, __ffma2_rn(my, my, c1));
        const float2 n2 = __ffma2_rn(make_float2(2.f, 2.f), sxy, c2);
        const float2 d2 = __fadd2_rn(__fadd2_rn(sxx, syy), c2);
        const float2 num = __fmul2_rn(n1, n2), den = __fmul2_rn(d1, d2);
        const float sa = __fdividef(num.x, den.x), sb = __fdividef(num.y, den.y);
        if (y < r_end) {
          if (x < I.mw) {
            sum += sa;
            if (MAP) P.map[I.map_off + int64_t(y) * I.mw + x] = sa;
          }
          if (x + 1 < I.mw) {
            sum += sb;
            if (MAP) P.map[I.map_off + int64_t(y) * I.mw + x + 1] = sb;
          }
        }
      }
    }
    __syncthreads();
  }
  // CTA reduction in binary64, one atomic per CTA
  double d = double(sum);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  __shared__ double red[kSsimThreads / 32];
  if ((tid & 31) == 0) red[tid >> 5] = d;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kSsimThreads / 32; ++w) t += red[w];
    atomicAdd(P.mssim + lo, t * I.inv_count);
  }
}

template <typename Smp, bool MAP>
tx16_status launch_ssim(const SsimImg* imgs, int n, const float* g, double* mssim, float* map, cudaStream_t st) {
  SsimParams<kSsimMaxImg> P;
  P.nimg = n;
  P.mssim = mssim;
  P.map = map;
  for (int k = 0; k < kWin; ++k) P.g[k] = g[k];
  int units = 0;
  for (int i = 0; i < n; ++i) {
    P.img[i] = imgs[i];
    P.img[i].unit0 = units;
    units += imgs[i].nstrips * ((imgs[i].mh + kSegRows - 1) / kSegRows);
  }
  P.nunits = units;
  static std::atomic<bool> attr{false};
  if (!attr) {
    if (cudaFuncSetAttribute(ssim_kernel<Smp, MAP, kSsimMaxImg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kSsimSmem)) != cudaSuccess)
      return TX16_ECUDA;
    attr = true;
  }
  ssim_kernel<Smp, MAP, kSsimMaxImg><<<units, kSsimThreads, kSsimSmem, st>>>(P);
  return cudaGetLastError() == cudaSuccess ? TX16_OK : TX16_ECUDA;
}

bool valid_ssim_image(const tx16_image& im) {
  if (im.data == nullptr || (reinterpret_cast<uintptr_t>(im.data) & 15u) != 0) return false;
  if (im.bits < 8 || im.bits > 12) return false;
  if (im.width < kWin || im.height < kWin) return false;
  if (im.pitch_bytes <= 0 || (im.pitch_bytes % 16) != 0) return false;
  if (im.pitch_bytes < int64_t(im.width) * sample_bytes(im.bits)) return false;
  // unit count and map offsets stay within int32 / int64
  const int64_t strips = (int64_t(im.width) - kHalo + kStripCols - 1) / kStripCols;
  const int64_t segs = (int64_t(im.height) - kHalo + kSegRows - 1) / kSegRows;
  return strips * segs < (int64_t(1) << 30);
}

}  // namespace
}  // namespace tx16

using namespace tx16;

extern "C" tx16_status tx16_ssim(const tx16_image* a, const tx16_image* b, int32_t n, double* mssim, float* map,
                                 void* stream) {
  TX16_TRACE("tx16_ssim");
  if (n < 0 || (n > 0 && (a == nullptr || b == nullptr || mssim == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(mssim) & 7u) != 0 || (reinterpret_cast<uintptr_t>(map) & 3u) != 0)
    return TX16_EINVAL;
  // the normalised 1-D window, formed in binary64 and rounded once
  double e[kWin], es = 0.0;
  for (int k = 0; k < kWin; ++k) {
    const double t = double(k - kHalo / 2);
    e[k] = std::exp(-t * t / (2.0 * 1.5 * 1.5));
    es += e[k];
  }
  float g[kWin];
  for (int k = 0; k < kWin; ++k) g[k] = float(e[k] / es);
  std::vector<SsimImg> I(n);
  int64_t map_off = 0;
  for (int i = 0; i < n; ++i) {
    if (!valid_ssim_image(a[i]) || !valid_ssim_image(b[i])) return TX16_EINVAL;
    if (a[i].width != b[i].width || a[i].height != b[i].height || a[i].bits != b[i].bits) return TX16_EINVAL;
    SsimImg& s = I[i];
    s.a = a[i].data;
    s.b = b[i].data;
    s.pa = a[i].pitch_bytes;
    s.pb = b[i].pitch_bytes;
    s.w = a[i].width;
    s.h = a[i].height;
    s.mw = s.w - kHalo;
    s.mh = s.h - kHalo;
    s.nstrips = (s.mw + kStripCols - 1) / kStripCols;
    s.map_off = map_off;
    map_off += int64_t(s.mw) * s.mh;
    s.inv_count = 1.0 / (double(s.mw) * double(s.mh));
    const double L = double((1 << a[i].bits) - 1);
    s.centre = float(1 << (a[i].bits - 1));
    s.c1 = float((0.01 * L) * (0.01 * L));
    s.c2 = float((0.03 * L) * (0.03 * L));
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(mssim, 0, sizeof(double) * size_t(n), st) != cudaSuccess) return TX16_ECUDA;
  int s = 0;
  while (s < n) {
    int e2 = s + 1;
    while (e2 < n && e2 - s < kSsimMaxImg && (a[e2].bits == 8) == (a[s].bits == 8)) ++e2;
    // map offsets are absolute: each launch gets the base map pointer
    tx16_status r;
    if (a[s].bits == 8)
      r = map ? launch_ssim<uint8_t, true>(I.data() + s, e2 - s, g, mssim + s, map, st)
              : launch_ssim<uint8_t, false>(I.data() + s, e2 - s, g, mssim + s, nullptr, st);
    else
      r = map ? launch_ssim<uint16_t, true>(I.data() + s, e2 - s, g, mssim + s, map, st)
              : launch_ssim<uint16_t, false>(I.data() + s, e2 - s, g, mssim + s, nullptr, st);
    if (r != TX16_OK) return r;
    s = e2;
  }
  return TX16_OK;
}
