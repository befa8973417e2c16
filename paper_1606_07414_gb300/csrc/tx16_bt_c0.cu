// One-block-per-thread codec, zonal class A (r <= 8): the kernels of
// tx16_fused_bt.cuh instantiated for this class alone, so that the classes
// compile in parallel.
#include "tx16_fused_bt.cuh"

namespace tx16 {

template tx16_status bt_batch<0>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_batch_keep<0>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_batch_ragged<0>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_list<0>(int, bool, const ImgParam*, int, int, unsigned*, int, int, unsigned long long*,
                                 cudaStream_t);
template int bt_list_ctas<0>(int, bool);
template void bt_variant_info<0>(int, int*, int*, int*);

}  // namespace tx16
