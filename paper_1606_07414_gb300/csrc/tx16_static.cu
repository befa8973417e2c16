// tx16_codec_batch_static: the work-list codec without any allocation.
//
// Some callers cannot allocate device memory at the point where they want to
// run the codec: a process whose whole card is handed to another allocator (a
// framework's caching pool sized to the device), a latency-critical loop in
// which cudaMalloc/cudaFree would synchronise the device, or a deployment that
// fixes its memory budget at start-up.  This entry point serves them: the work
// list the kernel needs (per-image descriptors and tile counters) lives in one
// fixed device array compiled into the library, instead of memory the library
// allocates (as tx16_plan_create does).  The caller still provides every input
// and output buffer.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (about 123 KB) until the process exits.  Host code cannot
// use the variable's name as a device address; the first call on each device
// looks the address up with cudaGetSymbolAddress (that device current) and
// keeps it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "tx16_internal.h"

namespace tx16 {
ImgParam make_param(const tx16_image& in, const tx16_image* out, const tx16_qparams& qp, int64_t blk0);
bool valid_qparams(const tx16_qparams& qp);
}  // namespace tx16

using namespace tx16;

namespace {

constexpr int kStaticMaxImages = 1024;  // TX16_STATIC_MAX_IMAGES in include/tx16.h
constexpr int kStaticRuns = 7;          // zone classes 0..5 + the general kernel

struct StaticWorkList {
  ImgParam table[kStaticMaxImages];
  unsigned counters[kStaticRuns];
};

static __device__ __align__(256) unsigned char g_static_work_list[sizeof(StaticWorkList)];

// The descriptors reach the device array through the parameters of a small
// kernel launched on the caller's stream (at most kUploadChunk per launch):
// kernel parameters are copied when the launch is issued, so the host
// staging below is free again as soon as the call returns and the call never
// waits for earlier work on the stream (a copy from pageable host memory
// would).
constexpr int kUploadChunk = 224;

struct UploadParams {
  int32_t offset;          // first table entry written
  int32_t count;           // entries in p
  int32_t clear;           // 1: also zero the tile counters and sse[0..nsse)
  int32_t nsse;
  unsigned long long* sse;  // device, or nullptr
  StaticWorkList* list;     // device address of g_static_work_list
  ImgParam p[kUploadChunk];
};
static_assert(sizeof(UploadParams) < 32000, "kernel parameters too large");
static_assert(sizeof(ImgParam) % 4 == 0, "descriptors copied as 32-bit words");

__global__ void static_upload_kernel(const __grid_constant__ UploadParams P) {
  const unsigned* src = reinterpret_cast<const unsigned*>(P.p);
  unsigned* dst = reinterpret_cast<unsigned*>(P.list->table + P.offset);
  const int words = P.count * int(sizeof(ImgParam) / 4);
  for (int w = int(threadIdx.x); w < words; w += int(blockDim.x)) dst[w] = src[w];
  if (P.clear) {
    if (threadIdx.x < unsigned(kStaticRuns)) P.list->counters[threadIdx.x] = 0u;
    if (P.sse != nullptr)
      for (int i = int(threadIdx.x); i < P.nsse; i += int(blockDim.x)) P.sse[i] = 0ull;
  }
}

std::mutex g_static_mu;                  // one call at a time builds and uploads the list
StaticWorkList* g_static_addr[64] = {};  // per device: address of g_static_work_list
ImgParam g_host_table[kStaticMaxImages]; // staging on the host (no heap allocation)
int g_host_class[kStaticMaxImages];
int64_t g_host_blk0[kStaticMaxImages];

tx16_status static_address(StaticWorkList** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TX16_ECUDA;
  if (g_static_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_work_list) != cudaSuccess || p == nullptr) return TX16_ECUDA;
    g_static_addr[dev] = static_cast<StaticWorkList*>(p);
  }
  *out = g_static_addr[dev];
  return TX16_OK;
}

}  // namespace

extern "C" tx16_status tx16_codec_batch_static(const tx16_image* in, const tx16_image* out, int32_t n,
                                               const tx16_qparams* qp, uint64_t* sse, int32_t* levels,
                                               void* stream) {
  TX16_TRACE("tx16_codec_batch_static");
  if (n < 0 || n > kStaticMaxImages) return TX16_EINVAL;  // beyond the fixed array
  if (n > 0 && (in == nullptr || qp == nullptr)) return TX16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(levels) & 15u) != 0 || (reinterpret_cast<uintptr_t>(sse) & 7u) != 0)
    return TX16_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!valid_image(in[i]) || !valid_qparams(qp[i])) return TX16_EINVAL;
    if (out != nullptr && (!valid_image(out[i]) || out[i].width != in[i].width ||
                           out[i].height != in[i].height || out[i].bits != in[i].bits))
      return TX16_EINVAL;
  }
  if (n == 0) return TX16_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticWorkList* dev = nullptr;
  const tx16_status as = static_address(&dev);
  if (as != TX16_OK) return as;

  // descriptors grouped by zone class (the general kernel's images last);
  // blk0 keeps each image's place in the caller's level layout
  int64_t blk0 = 0;
  for (int i = 0; i < n; ++i) {
    g_host_blk0[i] = blk0;
    blk0 += int64_t(in[i].width / 16) * (in[i].height / 16);
    const bool fast = in[i].bits == 8 && (qp[i].q <= 0.f || qp[i].q >= kFusedMinQ);
    if (fast) {
      const ImgParam p = make_param(in[i], out ? &out[i] : nullptr, qp[i], 0);
      g_host_class[i] = fused_zone_class(&p, 1);
    } else {
      g_host_class[i] = kStaticRuns - 1;
    }
  }
  int first[kStaticRuns] = {}, count[kStaticRuns] = {}, tiles[kStaticRuns] = {};
  int m = 0;
  for (int c = 0; c < kStaticRuns; ++c) {
    first[c] = m;
    for (int i = 0; i < n; ++i) {
      if (g_host_class[i] != c) continue;
      ImgParam p = make_param(in[i], out ? &out[i] : nullptr, qp[i], g_host_blk0[i]);
      p.out_index = i;
      p.tile0 = tiles[c];
      tiles[c] += (p.nblk + 15) / 16;
      g_host_table[m++] = p;
      ++count[c];
    }
  }
  // upload the list and clear what the kernels count from zero (see
  // static_upload_kernel)
  {
    UploadParams U;
    U.list = dev;
    U.sse = reinterpret_cast<unsigned long long*>(sse);
    U.nsse = n;
    for (int off = 0; off < m || off == 0; off += kUploadChunk) {
      U.offset = off;
      U.count = std::min(kUploadChunk, m - off);
      U.clear = off == 0 ? 1 : 0;
      std::memcpy(U.p, g_host_table + off, sizeof(ImgParam) * size_t(U.count));
      static_upload_kernel<<<1, 256, 0, st>>>(U);
      if (cudaGetLastError() != cudaSuccess) return TX16_ECUDA;
    }
  }
  unsigned long long* s64 = reinterpret_cast<unsigned long long*>(sse);
  for (int c = 0; c < kStaticRuns; ++c) {
    if (count[c] == 0) continue;
    tx16_status s = TX16_OK;
    if (c < kStaticRuns - 1) {
      s = launch_fused_list(c, levels != nullptr, out != nullptr, dev->table + first[c], count[c], tiles[c],
                            dev->counters + c, 1, 0, s64, levels, st);
    } else {
      for (int j = 0; j < count[c] && s == TX16_OK; ++j) {
        ImgParam q = g_host_table[first[c] + j];
        s = launch_blocks(kOpCodec, (q.flags & 0xff) == 8 ? 1 : 2, &q, 1, s64 ? s64 + q.out_index : nullptr,
                          levels, st);
      }
    }
    if (s != TX16_OK) return s;
  }
  return TX16_OK;
}
