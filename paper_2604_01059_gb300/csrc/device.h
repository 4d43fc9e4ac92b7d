// Device-side program cache and sampling entry points (device.cu).
#pragma once
#include <cstdint>

#include "program.h"

namespace tsim {

struct SampleArgs {
  uint64_t shots = 0, seed = 0, shot_offset = 0;
  uint64_t* meas = nullptr;
  uint64_t* det = nullptr;
  uint64_t* obs = nullptr;
  uint8_t* accept = nullptr;
};

void device_sample(const Program& p, const SampleArgs& a, void* stream);
void device_sample_batch(const Program* const* progs, int n, const SampleArgs* args, void* stream);
void device_sync(void* stream);
void device_release(DeviceProgram* d);

// exact monomial form of a Clifford factor value: value = 0 or sqrt2^s w^j
bool monomial_of(const ZW& v, int* zero, int* s, int* j);

}  // namespace tsim
