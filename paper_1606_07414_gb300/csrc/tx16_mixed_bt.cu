// The one-region-per-thread mixed 8/16 tiling kernel (tx16_mixed_bt.cuh):
// compiled class pairs (16x16 class, 8x8 class) and the dispatch to them.
#include "tx16_mixed_bt.cuh"

namespace tx16 {

template tx16_status mixed_bt_batch<0, 0>(const MixedParam*, int, unsigned long long*, uint8_t*, cudaStream_t);
template tx16_status mixed_bt_batch<1, 0>(const MixedParam*, int, unsigned long long*, uint8_t*, cudaStream_t);
template tx16_status mixed_bt_batch<1, 1>(const MixedParam*, int, unsigned long long*, uint8_t*, cudaStream_t);
template tx16_status mixed_bt_batch<2, 1>(const MixedParam*, int, unsigned long long*, uint8_t*, cudaStream_t);
template tx16_status mixed_bt_batch<3, 1>(const MixedParam*, int, unsigned long long*, uint8_t*, cudaStream_t);

namespace {
// Smallest 8x8 class whose column heights cover colh8 (-1: none).
int mix8_class(const uint8_t colh8[8]) {
  static const uint8_t H[2][8] = {{3, 1, 0, 0, 0, 0, 0, 0}, {5, 4, 3, 2, 1, 1, 0, 0}};
  for (int c = 0; c < 2; ++c) {
    bool in = true;
    for (int v = 0; v < 8; ++v) in = in && colh8[v] <= H[c][v];
    if (in) return c;
  }
  return -1;
}
}  // namespace

// Compiled pairs: 0 (A, 0), 1 (B, 0), 2 (B, 1), 3 (C, 1), 4 (D, 1); an image
// takes the first that covers both of its zones.
int mixed_bt_pair(const MixedParam& m) {
  const ImgParam& p = m.p;
  if ((p.flags & 0xff) != 8 || !(p.flags & kQuantFlag) || !fused_eligible(p) || p.dst == nullptr) return -1;
  const int c16 = fused_zone_class(&p, 1);
  const int c8 = mix8_class(m.colh8);
  if (c16 > 3 || c8 < 0) return -1;
  if (c8 == 0) return c16 <= 1 ? c16 : c16 + 1;
  return c16 <= 1 ? 2 : c16 + 1;
}

tx16_status launch_mixed_bt(int pair, const MixedParam* imgs, int n, unsigned long long* sse, uint8_t* split,
                            cudaStream_t stream) {
  if (n <= 0) return TX16_OK;
  switch (pair) {
    case 0: return mixed_bt_batch<0, 0>(imgs, n, sse, split, stream);
    case 1: return mixed_bt_batch<1, 0>(imgs, n, sse, split, stream);
    case 2: return mixed_bt_batch<1, 1>(imgs, n, sse, split, stream);
    case 3: return mixed_bt_batch<2, 1>(imgs, n, sse, split, stream);
    case 4: return mixed_bt_batch<3, 1>(imgs, n, sse, split, stream);
    default: return TX16_EINVAL;
  }
}

}  // namespace tx16
