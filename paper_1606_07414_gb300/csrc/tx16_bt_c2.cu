// One-block-per-thread codec, zonal class C (r <= 32): the kernels of
// tx16_fused_bt.cuh instantiated for this class alone, so that the classes
// compile in parallel.
#include "tx16_fused_bt.cuh"

namespace tx16 {

template tx16_status bt_batch<2>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_batch_keep<2>(bool, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_batch_ragged<2>(bool, int, const ImgParam*, int, unsigned long long*, cudaStream_t);
template tx16_status bt_list<2>(int, bool, const ImgParam*, int, int, unsigned*, int, int, unsigned long long*,
                                 cudaStream_t);
template int bt_list_ctas<2>(int, bool);
template void bt_variant_info<2>(int, int*, int*, int*);

}  // namespace tx16
