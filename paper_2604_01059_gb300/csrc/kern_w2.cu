// Sampling kernels for programs whose per-shot vector X is padded to 2
// 64-bit words (one translation unit per width, so the widths compile in
// parallel).
#include "kernels.cuh"

namespace tsim {

template cudaError_t launch_sample<2>(const LaunchArgs& a);
template cudaError_t launch_batch_group<2>(const BatchLaunchArgs& a);

}  // namespace tsim
