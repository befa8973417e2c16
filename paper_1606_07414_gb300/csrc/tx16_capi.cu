// C-ABI entry points of libtx16 (declared in include/tx16.h): argument
// checking, per-image parameter tables, and dispatch to the block kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "tx16_internal.h"

namespace tx16 {

int sample_bytes(int bits) { return bits == 8 ? 1 : 2; }

bool valid_image(const tx16_image& im) {
  if (im.data == nullptr) return false;
  if (im.bits < 8 || im.bits > 12) return false;
  if (im.width <= 0 || im.height <= 0 || (im.width % 16) != 0 || (im.height % 16) != 0) return false;
  const int64_t nblk = int64_t(im.width / 16) * int64_t(im.height / 16);
  if (nblk > (int64_t(1) << 30)) return false;
  if (im.pitch_bytes <= 0 || (im.pitch_bytes % 16) != 0) return false;
  if (im.pitch_bytes < int64_t(im.width) * sample_bytes(im.bits)) return false;
  if ((reinterpret_cast<uintptr_t>(im.data) & 15u) != 0) return false;
  return true;
}

// Zig-zag scan of a 16x16 block (JPEG convention, Sec. 3.1 zonal coding):
// anti-diagonals d = u + v in increasing order; odd d from row 0 downward,
// even d from the bottom row upward.  The cells of Z_r inside column v are
// always a prefix of rows (the scan finishes diagonal d before d + 1), so the
// zone is stored as 16 column heights.
void zonal_column_heights(int r, uint8_t colh[16]) {
  int rank[16][16];
  int k = 0;
  for (int d = 0; d <= 30; ++d) {
    const int ulo = d < 16 ? 0 : d - 15;
    const int uhi = d < 16 ? d : 15;
    if (d & 1) {
      for (int u = ulo; u <= uhi; ++u) rank[u][d - u] = k++;
    } else {
      for (int u = uhi; u >= ulo; --u) rank[u][d - u] = k++;
    }
  }
  for (int v = 0; v < 16; ++v) {
    int h = 0;
    for (int u = 0; u < 16; ++u) h += rank[u][v] < r ? 1 : 0;
    colh[v] = uint8_t(h);
  }
}

// s_u s_v = sqrt2^k / 16 with k = e(u) + e(v) (S of Sec. 2.1).  The quantiser
// with S merged in multiplies by f_k = fl32(s_u s_v / q) forward and by
// g_k = fl32(q s_u s_v) on the way back; both are formed in double first.
void quant_constants(float q, float f[5], float g[5]) {
  const double r2 = std::sqrt(2.0);
  const double dd[5] = {1.0, r2, 2.0, 2.0 * r2, 4.0};
  for (int k = 0; k < 5; ++k) {
    if (q > 0.f) {
      f[k] = float(dd[k] / (16.0 * double(q)));
      g[k] = float(double(q) * dd[k] / 16.0);
    } else {
      f[k] = 0.f;
      g[k] = 0.f;
    }
  }
}

bool valid_qparams(const tx16_qparams& qp) {
  return qp.r >= 1 && qp.r <= 256 && std::isfinite(qp.q);
}
static bool valid_qp(const tx16_qparams& qp) { return valid_qparams(qp); }

static void fill_quant(ImgParam& p, const tx16_qparams& qp) {
  quant_constants(qp.q, p.f, p.g);
  zonal_column_heights(qp.r, p.colh);
  if (qp.q > 0.f) p.flags |= kQuantFlag;
}

static ImgParam base_param(const tx16_image& im, int64_t blk0) {
  ImgParam p;
  std::memset(&p, 0, sizeof(p));
  p.src = im.data;
  p.src_pitch = im.pitch_bytes;
  p.blk0 = blk0;
  p.nbx = im.width / 16;
  p.nblk = (im.width / 16) * (im.height / 16);
  p.flags = im.bits;
  // m = floor(2^32 / nbx) (2^32 - 1 for nbx = 1): for blk < 2^31 the quotient
  // umulhi(blk, m) is exact or one too small, which the kernels correct
  p.out_index = 0;
  p.div_magic = p.nbx == 1 ? 0xFFFFFFFFu : uint32_t((uint64_t(1) << 32) / uint64_t(p.nbx));
  return p;
}

// Descriptor of one codec image: input, optional output, quantiser, and the
// index of its first block in the coefficient/level layout.
ImgParam make_param(const tx16_image& in, const tx16_image* out, const tx16_qparams& qp, int64_t blk0) {
  ImgParam p = base_param(in, blk0);
  if (out != nullptr) {
    p.dst = out->data;
    p.dst_pitch = out->pitch_bytes;
  }
  fill_quant(p, qp);
  return p;
}

// Launch runs of consecutive images with the same sample size together.
static tx16_status launch_runs(Op op, const tx16_image* imgs, std::vector<ImgParam>& P,
                               unsigned long long* sse, int32_t* coeffs, cudaStream_t stream) {
  const int n = int(P.size());
  int s = 0;
  while (s < n) {
    int e = s + 1;
    while (e < n && sample_bytes(imgs[e].bits) == sample_bytes(imgs[s].bits)) ++e;
    const tx16_status st = launch_blocks(op, sample_bytes(imgs[s].bits), P.data() + s, e - s,
                                         sse ? sse + s : nullptr, coeffs, stream);
    if (st != TX16_OK) return st;
    s = e;
  }
  return TX16_OK;
}

}  // namespace tx16

using namespace tx16;

namespace tx16 {

// Runs of consecutive images by kernel: the fused 8-bit kernels (steps of
// q >= kFusedMinQ or no quantiser), the fused 16-bit path (9..12-bit samples
// with a quantiser of q >= 2^(bits-8) kFusedMinQ), the general block kernel
// for the rest.  sse[i] belongs to P[i]; levels (or null) are block-major in
// the order of P.
tx16_status launch_codec_runs(ImgParam* P, int n, unsigned long long* sse, int32_t* levels, cudaStream_t st) {
  auto kind = [&](const ImgParam& p) {
    if ((p.flags & 0xff) == 8) return fused_eligible(p) ? 1 : 0;
    return fused_bt16_eligible(p) ? 2 : 0;
  };
  int s = 0;
  while (s < n) {
    const int ks = kind(P[s]);
    const int sb = sample_bytes(P[s].flags & 0xff);
    int e = s + 1;
    while (e < n && kind(P[e]) == ks && sample_bytes(P[e].flags & 0xff) == sb) ++e;
    unsigned long long* ss = sse ? sse + s : nullptr;
    const tx16_status r = ks == 1   ? launch_fused_u8(P + s, e - s, ss, levels, st)
                          : ks == 2 ? launch_fused_u16(P + s, e - s, ss, levels, st)
                                    : launch_blocks(kOpCodec, sb, P + s, e - s, ss, levels, st);
    if (r != TX16_OK) return r;
    s = e;
  }
  return TX16_OK;
}

}  // namespace tx16

extern "C" {

const char* tx16_status_str(tx16_status s) {
  switch (s) {
    case TX16_OK: return "ok";
    case TX16_EINVAL: return "invalid argument";
    case TX16_ENOMEM: return "out of memory";
    case TX16_ECUDA: return "CUDA error";
    case TX16_ETIMEOUT: return "timed out";
    case TX16_EBUSY: return "busy";
  }
  return "unknown status";
}

int64_t tx16_image_blocks(const tx16_image* img) {
  if (img == nullptr || !valid_image(*img)) return -1;
  return int64_t(img->width / 16) * int64_t(img->height / 16);
}

tx16_status tx16_forward(const tx16_image* imgs, int32_t n, int32_t* coeffs, void* stream) {
  TX16_TRACE("tx16_forward");
  if (n < 0 || (n > 0 && (imgs == nullptr || coeffs == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(coeffs) & 15u) != 0) return TX16_EINVAL;
  std::vector<ImgParam> P(n);
  int64_t blk0 = 0;
  for (int i = 0; i < n; ++i) {
    if (!valid_image(imgs[i])) return TX16_EINVAL;
    P[i] = base_param(imgs[i], blk0);
    blk0 += P[i].nblk;
  }
  if (n == 0) return TX16_OK;
  return launch_runs(kOpForward, imgs, P, nullptr, coeffs, static_cast<cudaStream_t>(stream));
}

tx16_status tx16_quantise(const int32_t* coeffs, int64_t nblk, tx16_qparams qp, int32_t* levels,
                          void* stream) {
  TX16_TRACE("tx16_quantise");
  if (nblk < 0 || !valid_qp(qp)) return TX16_EINVAL;
  if (nblk == 0) return TX16_OK;
  if (coeffs == nullptr || levels == nullptr) return TX16_EINVAL;
  if (((reinterpret_cast<uintptr_t>(coeffs) | reinterpret_cast<uintptr_t>(levels)) & 15u) != 0)
    return TX16_EINVAL;
  ImgParam p;
  std::memset(&p, 0, sizeof(p));
  fill_quant(p, qp);
  return launch_quantise(coeffs, nblk, p, levels, static_cast<cudaStream_t>(stream));
}

tx16_status tx16_inverse(const int32_t* levels, const tx16_image* out, int32_t n, const tx16_qparams* qp,
                         void* stream) {
  TX16_TRACE("tx16_inverse");
  if (n < 0 || (n > 0 && (levels == nullptr || out == nullptr || qp == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(levels) & 15u) != 0) return TX16_EINVAL;
  std::vector<ImgParam> P(n);
  int64_t blk0 = 0;
  for (int i = 0; i < n; ++i) {
    if (!valid_image(out[i]) || !valid_qp(qp[i])) return TX16_EINVAL;
    P[i] = base_param(out[i], blk0);
    P[i].src = nullptr;
    P[i].dst = out[i].data;
    P[i].dst_pitch = out[i].pitch_bytes;
    fill_quant(P[i], qp[i]);
    blk0 += P[i].nblk;
  }
  if (n == 0) return TX16_OK;
  return launch_runs(kOpInverse, out, P, nullptr, const_cast<int32_t*>(levels),
                     static_cast<cudaStream_t>(stream));
}

tx16_status tx16_codec_batch(const tx16_image* in, const tx16_image* out, int32_t n, const tx16_qparams* qp,
                             uint64_t* sse, int32_t* levels, void* stream) {
  TX16_TRACE("tx16_codec_batch");
  if (n < 0 || (n > 0 && (in == nullptr || qp == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(levels) & 15u) != 0 || (reinterpret_cast<uintptr_t>(sse) & 7u) != 0)
    return TX16_EINVAL;
  std::vector<ImgParam> P(n);
  int64_t blk0 = 0;
  for (int i = 0; i < n; ++i) {
    if (!valid_image(in[i]) || !valid_qp(qp[i])) return TX16_EINVAL;
    if (out != nullptr) {
      if (!valid_image(out[i]) || out[i].width != in[i].width || out[i].height != in[i].height ||
          out[i].bits != in[i].bits)
        return TX16_EINVAL;
    }
    P[i] = base_param(in[i], blk0);
    if (out != nullptr) {
      P[i].dst = out[i].data;
      P[i].dst_pitch = out[i].pitch_bytes;
    }
    fill_quant(P[i], qp[i]);
    blk0 += P[i].nblk;
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sse != nullptr && cudaMemsetAsync(sse, 0, sizeof(uint64_t) * size_t(n), st) != cudaSuccess)
    return TX16_ECUDA;
  unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sse);
  return launch_codec_runs(P.data(), n, s64, levels, st);
}

tx16_status tx16_sse(const tx16_image* a, const tx16_image* b, int32_t n, uint64_t* sse, void* stream) {
  TX16_TRACE("tx16_sse");
  if (n < 0 || (n > 0 && (a == nullptr || b == nullptr || sse == nullptr))) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(sse) & 7u) != 0) return TX16_EINVAL;
  std::vector<ImgParam> P(n);
  for (int i = 0; i < n; ++i) {
    if (!valid_image(a[i]) || !valid_image(b[i]) || a[i].width != b[i].width || a[i].height != b[i].height ||
        a[i].bits != b[i].bits)
      return TX16_EINVAL;
    P[i] = base_param(a[i], 0);
    P[i].dst = b[i].data;
    P[i].dst_pitch = b[i].pitch_bytes;
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(sse, 0, sizeof(uint64_t) * size_t(n), st) != cudaSuccess) return TX16_ECUDA;
  return launch_runs(kOpSse, a, P, reinterpret_cast<unsigned long long*>(sse), nullptr, st);
}

tx16_status tx16_psnr(const uint64_t* sse, const tx16_image* imgs, int32_t n, double* psnr) {
  if (n < 0 || (n > 0 && (sse == nullptr || imgs == nullptr || psnr == nullptr))) return TX16_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (imgs[i].bits < 8 || imgs[i].bits > 12 || imgs[i].width <= 0 || imgs[i].height <= 0)
      return TX16_EINVAL;
    const double peak = double((1 << imgs[i].bits) - 1);
    psnr[i] = sse[i] == 0 ? HUGE_VAL
                          : 10.0 * std::log10(peak * peak * double(imgs[i].width) * double(imgs[i].height) /
                                              double(sse[i]));
  }
  return TX16_OK;
}

}  // extern "C"
