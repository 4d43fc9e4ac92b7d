// Sampling kernels for programs whose per-shot vector X is padded to 8
// 64-bit words (one translation unit per width, so the widths compile in
// parallel).
#include "kernels.cuh"

namespace tsim {

template cudaError_t launch_sample<8>(const LaunchArgs& a);
template cudaError_t launch_batch_group<8>(const BatchLaunchArgs& a);

}  // namespace tsim
