// Source iteration with the angular sum of Eq. 12 on the tcgen05 tensor cores (BF16 in,
// FP32 accumulate in tensor memory).
#include <cstdint>

#include "device.cuh"

namespace trinity {

bool scatter_bf16_supported(int na) { (void)na; return false; }

cudaError_t launch_scatter_bf16(const GridParams&, const DirInfo*, const uint16_t*, const float*,
                                const float*, const float*, const float*, float*, float*, float,
                                int, RunState, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace trinity
