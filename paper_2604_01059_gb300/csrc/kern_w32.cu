// Sampling kernels for programs whose per-shot vector X is padded to 32
// 64-bit words (one translation unit per width, so the widths compile in
// parallel).
#include "kernels.cuh"

namespace tsim {

template cudaError_t launch_sample<32>(const LaunchArgs& a);
template cudaError_t launch_batch_group<32>(const BatchLaunchArgs& a);

}  // namespace tsim
