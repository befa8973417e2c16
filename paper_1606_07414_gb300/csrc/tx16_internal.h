// Internal types shared by the libtx16 translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "tx16.h"

namespace tx16 {

// An NVTX range over one C-ABI call or serving stage, named after it, so that
// profiler timelines (nsys, ncu --nvtx) group kernels by the call that issued
// them.  NVTX v3 is header-only: without an attached tool a push or pop is a
// call through an empty slot.
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};
#define TX16_TRACE(name) ::tx16::Trace tx16_trace_range_(name)

constexpr int kTileBlocks = 16;            // 16x16 blocks per CTA iteration
constexpr int kThreads = 16 * kTileBlocks;  // one thread per block row
constexpr int kQuantFlag = 1 << 8;          // ImgParam::flags: q > 0

// Everything a kernel needs to know about one image, passed by value in the
// launch parameters (no device-side descriptor table, no allocation).
struct ImgParam {
  const void* src;     // samples read (forward / codec) -- device
  void* dst;           // samples written (codec / inverse) or nullptr -- device
  int64_t src_pitch;   // bytes
  int64_t dst_pitch;   // bytes
  int64_t blk0;        // index of the image's first block in the coefficient buffer
  int32_t nbx;         // blocks per block row (width / 16)
  int32_t nblk;        // blocks in the image
  int32_t tile0;       // first tile of this image within the launch
  int32_t flags;       // bits (low 8) | kQuantFlag
  uint32_t div_magic;  // blk / nbx = umulhi(blk, div_magic), or one more
  int32_t out_index;   // index of this image's SSE in the caller's sse[] array
  float f[5];          // fl32(sqrt2^k / (16 q)), k = e(u) + e(v)   (forward scale)
  float g[5];          // fl32(q sqrt2^k / 16)                      (inverse scale)
  uint8_t colh[16];    // kept rows of column v: |Z_r ∩ column v| (a prefix 0..colh-1)
};

template <int MAXI>
struct BatchParams {
  int32_t nimg;
  int32_t ntiles;
  unsigned long long* sse;  // per image of this launch (already offset), or nullptr
  int32_t* coeffs;          // forward: output; inverse: input; codec: levels or nullptr
  ImgParam img[MAXI];
};

// Largest per-launch image count; sizeof(BatchParams<kMaxImg>) must stay under
// the 32 KB kernel-parameter limit.
constexpr int kMaxImg = 256;
static_assert(sizeof(BatchParams<kMaxImg>) < 32000, "kernel parameters too large");

enum Op { kOpForward = 0, kOpCodec = 1, kOpInverse = 2, kOpSse = 3 };

// Host helpers (tx16_host.cpp)
bool valid_image(const tx16_image& im);
int sample_bytes(int bits);
void zonal_column_heights(int r, uint8_t colh[16]);
void quant_constants(float q, float f[5], float g[5]);

// Fused 8-bit codec (tx16_fused.cu): needs q >= kFusedMinQ when quantising
// (|Y f| + 1/2 < 2^23 keeps the rounding trick exact).
constexpr float kFusedMinQ = 1.0f / 256.0f;
tx16_status launch_fused_u8(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                            cudaStream_t stream);
int fused_zone_class(const ImgParam* imgs, int n);  // 0..5: r_max 8, 16, 32, 64, 128, 256
bool fused_eligible(const ImgParam& p);  // 8-bit samples and q >= kFusedMinQ (or no q)
// Work-list launch: descriptors in device memory (tile0 relative to the list,
// ascending), tiles claimed `chunk` at a time from *counter (zeroed before).
tx16_status launch_fused_list(int zone, bool lev, bool dst, const ImgParam* d_imgs, int nimg, int ntiles,
                              unsigned* counter, int chunk, int ctas_per_sm, unsigned long long* sse,
                              int32_t* levels, cudaStream_t stream);
int fused_list_max_ctas(int zone, bool lev, bool dst);  // resident CTAs per SM
// One-block-per-thread fused kernel (tx16_fused_bt.cu): zonal classes with at
// most 8 kept columns, no level output.
bool fused_bt_supports(int zone, bool levels);
tx16_status launch_fused_bt(int zone, bool dst, const ImgParam* imgs, int n, unsigned long long* sse,
                            cudaStream_t stream);
// The same over images whose out_index are their SSE slots of sse (at most
// kMaxImg): a subset of a call's images, grouped by class.
tx16_status launch_fused_bt_grouped(int zone, bool dst, const ImgParam* imgs, int n, unsigned long long* sse,
                                    cudaStream_t stream);
// Its work-list form: descriptors in device memory with tile0 in warp tiles
// of 32 blocks (bt_warp_tiles), relative to the list and ascending; warps
// claim `chunk` tiles at a time from *counter (zeroed before the launch).
// Each class has fused_bt_variants() compiled configurations (variant 0:
// the default; the plan autotuner times the others).
int bt_warp_tiles(int nblk);
int bt_class_rmax(int zone);           // largest r of zonal class `zone` (0..5)
int fused_bt_warps_per_cta(int zone);  // warps per CTA of the one-block-per-thread kernel (variant 0)
int fused_bt_variants(int zone);       // compiled configurations of the work-list kernel (0: none)
void fused_bt_variant_info(int zone, int variant, int* warps, int* park, int* stages);
tx16_status launch_fused_bt_list(int zone, int variant, bool dst, const ImgParam* d_imgs, int nimg, int ntiles,
                                 unsigned* counter, int chunk, int ctas_per_sm, unsigned long long* sse,
                                 cudaStream_t stream);
int fused_bt_list_max_ctas(int zone, int variant, bool dst);  // resident CTAs per SM
// Images whose height is not a multiple of 16 (tx16_codec_any_size), coded
// whole by the one-block-per-thread kernel: the descriptor covers the padded
// block rows, flags bits 12..15 hold the rows missing from the last block row
// (kBtMissingShift); rows below the image repeat its last row, and only the
// image's rows are written and counted in sse[out_index].
constexpr int kBtMissingShift = 12;
bool fused_bt_ragged_supports(const ImgParam& p);
tx16_status launch_fused_bt_ragged(const ImgParam* imgs, int n, unsigned long long* sse, cudaStream_t stream);
// 9..12-bit planes (uint16 samples) with a quantiser of q >= 2^(bits-8)/256:
// the one-block-per-thread kernel for zonal classes up to 8 kept columns and
// no levels, the general kernel otherwise.
bool fused_bt16_eligible(const ImgParam& p);
tx16_status launch_fused_u16(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                             cudaStream_t stream);

// Mixed 8/16 tiling (tx16_mixed.cu): per image, the 16x16 quantiser and
// region grid (p; blk0 = first region in the split map, out_index = SSE
// slot), the 8x8 quantiser (S8 merged: f8 = fl32(2^(-3+k/2) / q), g8 =
// fl32(q 2^(-3+k/2))), the kept rows of each 8x8 column and the tiling mode
// (0 automatic, 1 all 16x16, 2 all 8x8).
struct MixedParam {
  ImgParam p;
  float f8[5];
  float g8[5];
  uint8_t colh8[8];
  int32_t mode;
};
constexpr int kMixMaxImg = 160;  // images per launch (kernel-parameter limit)
// The one-region-per-thread kernel (tx16_mixed_bt.cu): 8-bit samples with a
// quantiser of q >= kFusedMinQ, an output plane, 16x16 zones of r <= 64 and
// 8x8 zones of r8 <= 16.  mixed_bt_pair: the compiled class pair that covers
// the image (0..4), or -1; one launch takes images of one pair.
constexpr int kMixBtPairs = 5;
int mixed_bt_pair(const MixedParam& m);
tx16_status launch_mixed_bt(int pair, const MixedParam* imgs, int n, unsigned long long* sse, uint8_t* split,
                            cudaStream_t stream);

// Launchers (tx16_codec.cu).  `imgs` points at `n` ImgParam already filled in
// (except tile0, set here), all with the same sample size.
tx16_status launch_blocks(Op op, int sample_bytes, ImgParam* imgs, int n,
                          unsigned long long* sse, int32_t* coeffs, cudaStream_t stream);
tx16_status launch_quantise(const int32_t* coeffs, int64_t nblk, const ImgParam& qp,
                            int32_t* levels, cudaStream_t stream);

int device_sm_count();

// The codec over n images by runs of the kernel that suits them (fused 8-bit,
// fused 16-bit, general); tx16_capi.cu.
tx16_status launch_codec_runs(ImgParam* P, int n, unsigned long long* sse, int32_t* levels, cudaStream_t st);

}  // namespace tx16
