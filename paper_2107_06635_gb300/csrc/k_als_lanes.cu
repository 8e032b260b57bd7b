// Instantiations of the ALS kernel k_als with the lane build of the reduced metric only
// (one CTA per item at two or three CTAs per SM, or a cluster per item).
#include "als_kernel.cuh"

namespace ntu {

cudaError_t als_launch_lanes(const AlsArgs& a, int n, int split, bool three, size_t smem,
                             cudaStream_t stream) {
  return als_launch_impl<0>(a, n, split, three, smem, stream);
}

}  // namespace ntu
