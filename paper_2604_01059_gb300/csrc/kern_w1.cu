// Sampling kernels for programs whose per-shot vector X is padded to 1
// 64-bit word (one translation unit per width, so the widths compile in
// parallel).
#include "kernels.cuh"

namespace tsim {

template cudaError_t launch_sample<1>(const LaunchArgs& a);
template cudaError_t launch_batch_group<1>(const BatchLaunchArgs& a);

}  // namespace tsim
