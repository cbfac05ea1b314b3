// Run-time model-specialised builds of the batched kernels (shac_jit.cu).
#pragma once
#include <string>
#include <vector>

#include "../../include/shacsim.h"
#include "shac_kernels.cuh"

namespace shac {

// The forward (k_batched<false>) and adjoint (k_batched<true>) kernels of one
// build, as handles the runtime's launch and attribute calls accept, and the
// key the launch arguments must carry (BatchedArgs::spec_key).
struct JitKernels {
  const void* fwd = nullptr;
  const void* adj = nullptr;
  unsigned int key = 0;
};

// Build (or fetch from the process-wide cache) the kernels for model layout m
// and link parents `parent` (m.L entries) on `device` with team size `lanes`,
// register dense row capacity `rows` (0: the shared-memory dense stages) and
// per-environment scratch stride `stride`.  SHAC_ERR_CUDA if the run-time
// compiler or the module load fails (the compiler's log in *log when given).
shac_status jit_kernels(int device, const DevModel& m, const std::vector<int>& parent, int lanes, int rows,
                        int stride, JitKernels* out, std::string* log);

}  // namespace shac
