// Dispatch of the one-block-per-thread codec (tx16_fused_bt.cuh) over its
// zonal classes; each class is compiled in its own translation unit
// (tx16_bt_c<class>.cu) so that the classes build in parallel.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "tx16_fused_bt.cuh"
#include "tx16_internal.h"

namespace tx16 {

extern template tx16_status bt_batch_keep<0>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_keep<1>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_keep<2>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_keep<3>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_keep<4>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_keep<5>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch<0>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch<1>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch<2>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch<3>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_ragged<0>(bool, int, const ImgParam*, int, unsigned long long*,
                                                cudaStream_t);
extern template tx16_status bt_batch_ragged<1>(bool, int, const ImgParam*, int, unsigned long long*,
                                                cudaStream_t);
extern template tx16_status bt_batch_ragged<2>(bool, int, const ImgParam*, int, unsigned long long*,
                                                cudaStream_t);
extern template tx16_status bt_batch_ragged<3>(bool, int, const ImgParam*, int, unsigned long long*,
                                                cudaStream_t);
extern template tx16_status bt_list<0>(int, bool, const ImgParam*, int, int, unsigned*, int, int,
                                       unsigned long long*, cudaStream_t);
extern template tx16_status bt_list<1>(int, bool, const ImgParam*, int, int, unsigned*, int, int,
                                       unsigned long long*, cudaStream_t);
extern template tx16_status bt_list<2>(int, bool, const ImgParam*, int, int, unsigned*, int, int,
                                       unsigned long long*, cudaStream_t);
extern template tx16_status bt_list<3>(int, bool, const ImgParam*, int, int, unsigned*, int, int,
                                       unsigned long long*, cudaStream_t);
extern template int bt_list_ctas<0>(int, bool);
extern template void bt_variant_info<0>(int, int*, int*, int*);
extern template int bt_list_ctas<1>(int, bool);
extern template void bt_variant_info<1>(int, int*, int*, int*);
extern template int bt_list_ctas<2>(int, bool);
extern template void bt_variant_info<2>(int, int*, int*, int*);
extern template int bt_list_ctas<3>(int, bool);
extern template void bt_variant_info<3>(int, int*, int*, int*);
extern template tx16_status bt_batch<4>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_ragged<4>(bool, int, const ImgParam*, int, unsigned long long*,
                                                cudaStream_t);
extern template tx16_status bt_list<4>(int, bool, const ImgParam*, int, int, unsigned*, int, int,
                                       unsigned long long*, cudaStream_t);
extern template int bt_list_ctas<4>(int, bool);
extern template void bt_variant_info<4>(int, int*, int*, int*);
extern template tx16_status bt_batch<5>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
extern template tx16_status bt_batch_ragged<5>(bool, int, const ImgParam*, int, unsigned long long*,
                                                cudaStream_t);
extern template tx16_status bt_list<5>(int, bool, const ImgParam*, int, int, unsigned*, int, int,
                                       unsigned long long*, cudaStream_t);
extern template int bt_list_ctas<5>(int, bool);
extern template void bt_variant_info<5>(int, int*, int*, int*);

// Zonal classes routed to this kernel for 8-bit samples (bit c for class c;
// compile-time tunable): all six.  With each warp on a contiguous run of
// tiles, classes E and F run faster here than on the two-blocks-per-pair
// kernel (r = 128: 5539 against 4163 Mblocks/s, r = 256: 4359 against 4142);
// with tiles w, w + W, ... they had measured slower (3929 and 3474).
// 9..12-bit samples: A..C.
#ifndef TX16_BT_ZONE_MASK
#define TX16_BT_ZONE_MASK 0x3f
#endif

bool fused_bt_supports(int zone, bool levels) {
  return !levels && zone >= 0 && zone < kBtClasses && ((TX16_BT_ZONE_MASK >> zone) & 1);
}

int bt_class_rmax(int zone) {
  switch (zone) {
    case 0: return BtClass<0>::kRmax;
    case 1: return BtClass<1>::kRmax;
    case 2: return BtClass<2>::kRmax;
    case 3: return BtClass<3>::kRmax;
    case 4: return BtClass<4>::kRmax;
    default: return BtClass<5>::kRmax;
  }
}

int bt_warp_tiles(int nblk) { return (nblk + kWarpTile - 1) / kWarpTile; }

int fused_bt_warps_per_cta(int zone) {
  switch (zone) {
    case 0: return BtLimits<0>::kWarps;
    case 1: return BtLimits<1>::kWarps;
    case 2: return BtLimits<2>::kWarps;
    case 3: return BtLimits<3>::kWarps;
    case 4: return BtLimits<4>::kWarps;
    default: return BtLimits<5>::kWarps;
  }
}

tx16_status launch_fused_bt_list(int zone, int variant, bool dst, const ImgParam* d_imgs, int nimg, int ntiles,
                                 unsigned* counter, int chunk, int ctas_per_sm, unsigned long long* sse,
                                 cudaStream_t stream) {
  switch (zone) {
    case 0: return bt_list<0>(variant, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 1: return bt_list<1>(variant, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 2: return bt_list<2>(variant, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 3: return bt_list<3>(variant, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 4: return bt_list<4>(variant, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    case 5: return bt_list<5>(variant, dst, d_imgs, nimg, ntiles, counter, chunk, ctas_per_sm, sse, stream);
    default: return TX16_EINVAL;
  }
}

int fused_bt_list_max_ctas(int zone, int variant, bool dst) {
  switch (zone) {
    case 0: return bt_list_ctas<0>(variant, dst);
    case 1: return bt_list_ctas<1>(variant, dst);
    case 2: return bt_list_ctas<2>(variant, dst);
    case 3: return bt_list_ctas<3>(variant, dst);
    case 4: return bt_list_ctas<4>(variant, dst);
    case 5: return bt_list_ctas<5>(variant, dst);
    default: return 0;
  }
}

int fused_bt_variants(int zone) { return fused_bt_supports(zone, false) ? kBtVariants : 0; }

void fused_bt_variant_info(int zone, int variant, int* warps, int* park, int* stages) {
  switch (zone) {
    case 0: bt_variant_info<0>(variant, warps, park, stages); break;
    case 1: bt_variant_info<1>(variant, warps, park, stages); break;
    case 2: bt_variant_info<2>(variant, warps, park, stages); break;
    case 3: bt_variant_info<3>(variant, warps, park, stages); break;
    case 4: bt_variant_info<4>(variant, warps, park, stages); break;
    case 5: bt_variant_info<5>(variant, warps, park, stages); break;
    default: *warps = *park = *stages = 0; break;
  }
}

tx16_status launch_fused_bt(int zone, bool dst, const ImgParam* imgs, int n, unsigned long long* sse,
                            cudaStream_t stream) {
  switch (zone) {
    case 0: return bt_batch<0>(dst, 1, imgs, n, sse, stream);
    case 1: return bt_batch<1>(dst, 1, imgs, n, sse, stream);
    case 2: return bt_batch<2>(dst, 1, imgs, n, sse, stream);
    case 3: return bt_batch<3>(dst, 1, imgs, n, sse, stream);
    case 4: return bt_batch<4>(dst, 1, imgs, n, sse, stream);
    case 5: return bt_batch<5>(dst, 1, imgs, n, sse, stream);
    default: return TX16_EINVAL;
  }
}

tx16_status launch_fused_bt_grouped(int zone, bool dst, const ImgParam* imgs, int n, unsigned long long* sse,
                                    cudaStream_t stream) {
  switch (zone) {
    case 0: return bt_batch_keep<0>(dst, imgs, n, sse, stream);
    case 1: return bt_batch_keep<1>(dst, imgs, n, sse, stream);
    case 2: return bt_batch_keep<2>(dst, imgs, n, sse, stream);
    case 3: return bt_batch_keep<3>(dst, imgs, n, sse, stream);
    case 4: return bt_batch_keep<4>(dst, imgs, n, sse, stream);
    case 5: return bt_batch_keep<5>(dst, imgs, n, sse, stream);
    default: return TX16_EINVAL;
  }
}

tx16_status launch_fused_bt_ragged(const ImgParam* imgs, int n, unsigned long long* sse, cudaStream_t stream) {
  // runs of equal sample size and zonal class, at most kMaxImg per launch
  std::vector<ImgParam> run;
  for (int sb = 1; sb <= 2; ++sb) {
    for (int zone = 0; zone < kBtClasses; ++zone) {
      run.clear();
      for (int i = 0; i < n; ++i)
        if (sample_bytes(imgs[i].flags & 0xff) == sb && fused_zone_class(&imgs[i], 1) == zone) run.push_back(imgs[i]);
      for (size_t s = 0; s < run.size(); s += kMaxImg) {
        const int m = int(std::min<size_t>(kMaxImg, run.size() - s));
        const bool dst = run[s].dst != nullptr;
        tx16_status st;
        switch (zone) {
          case 0: st = bt_batch_ragged<0>(dst, sb, run.data() + s, m, sse, stream); break;
          case 1: st = bt_batch_ragged<1>(dst, sb, run.data() + s, m, sse, stream); break;
          case 2: st = bt_batch_ragged<2>(dst, sb, run.data() + s, m, sse, stream); break;
          case 3: st = bt_batch_ragged<3>(dst, sb, run.data() + s, m, sse, stream); break;
          case 4: st = bt_batch_ragged<4>(dst, sb, run.data() + s, m, sse, stream); break;
          default: st = bt_batch_ragged<5>(dst, sb, run.data() + s, m, sse, stream); break;
        }
        if (st != TX16_OK) return st;
      }
    }
  }
  return TX16_OK;
}

bool fused_bt_ragged_supports(const ImgParam& p) {
  const int bits = p.flags & 0xff;
  const int zone = fused_zone_class(&p, 1);
  if (bits == 8) return fused_eligible(p) && fused_bt_supports(zone, false);
  return fused_bt16_eligible(p) && zone <= 2;
}

bool fused_bt16_eligible(const ImgParam& p) {
  const int bits = p.flags & 0xff;
  // a quantiser (the exact no-quantiser inverse needs the integer kernel
  // beyond 8 bits) with |Y f| + 1/2 < 2^23 for the rounding trick:
  // q >= 2^(bits - 8) / 256
  return bits > 8 && bits <= 12 && (p.flags & kQuantFlag) && p.g[0] * 16.0f >= kFusedMinQ * float(1 << (bits - 8));
}

tx16_status launch_fused_u16(const ImgParam* imgs, int n, unsigned long long* sse, int32_t* levels,
                             cudaStream_t stream) {
  for (int s = 0; s < n; s += kMaxImg) {
    const int m = std::min(kMaxImg, n - s);
    const int zone = fused_zone_class(imgs + s, m);
    const bool dst = imgs[s].dst != nullptr;
    ImgParam* mut = const_cast<ImgParam*>(imgs + s);
    unsigned long long* ss = sse ? sse + s : nullptr;
    tx16_status st;
    if (zone <= 2 && levels == nullptr) {
      st = zone == 0 ? bt_batch<0>(dst, 2, imgs + s, m, ss, stream)
                     : (zone == 1 ? bt_batch<1>(dst, 2, imgs + s, m, ss, stream)
                                  : bt_batch<2>(dst, 2, imgs + s, m, ss, stream));
    } else {
      st = launch_blocks(kOpCodec, 2, mut, m, ss, levels, stream);
    }
    if (st != TX16_OK) return st;
  }
  return TX16_OK;
}

}  // namespace tx16
