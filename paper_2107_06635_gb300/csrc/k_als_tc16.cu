// Instantiations of the ALS kernel k_als with the tensor-core build of the reduced metric at K = D r = 16
// (one CTA per item at two or three CTAs per SM, or a cluster per item).
#include "als_kernel.cuh"

namespace ntu {

cudaError_t als_launch_tc16(const AlsArgs& a, int n, int split, bool three, size_t smem,
                            cudaStream_t stream) {
  return als_launch_impl<16>(a, n, split, three, smem, stream);
}

}  // namespace ntu
