// One-block-per-thread codec, zonal class D (r <= 64): the kernels of
// tx16_fused_bt.cuh instantiated for this class alone, so that the classes
// compile in parallel.
#include "tx16_fused_bt.cuh"

namespace tx16 {

template tx16_status bt_batch<3>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_batch_keep<3>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_batch_ragged<3>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_list<3>(int, bool, const ImgParam*, int, int, unsigned*, int, int, unsigned long long*,
                                 cudaStream_t);
template int bt_list_ctas<3>(int, bool);
template void bt_variant_info<3>(int, int*, int*, int*);

}  // namespace tx16
