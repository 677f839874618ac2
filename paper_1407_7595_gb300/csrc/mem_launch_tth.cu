// Kernel instantiations for the dilepton ttH process (fixed-budget integration and
// point evaluation; one build for parametric and tabulated PDFs, as for dilepton
// ttbar: the FP64 neutrino solution and the production amplitude dominate).
#include "mem_launch.cuh"
#include "mem_launch_config.h"
#include "mem_tth.cuh"

namespace mem {

// The ttH kernels keep up to ~1.5 KB per thread on the stack (the out-of-line FP64
// solver stages and the spinor chains); make sure the context's per-thread stack
// limit covers it before their first launch.
cudaError_t prepare_tth() {
  size_t cur = 0;
  cudaError_t e = cudaDeviceGetLimit(&cur, cudaLimitStackSize);
  if (e == cudaSuccess && cur < 2048) e = cudaDeviceSetLimit(cudaLimitStackSize, 2048);
  return e;
}

cudaError_t launch_integrate_tth(const IntegrateArgs& a, cudaStream_t st) {
  cudaError_t e = prepare_tth();
  if (e != cudaSuccess) return e;
  return run_integrate<PhysTTH, PPT_DL, MINB_TH, MINB_TH_MAIN>(a, st);
}
cudaError_t launch_eval_tth(const EvalArgs& a, cudaStream_t st) {
  cudaError_t e = prepare_tth();
  if (e != cudaSuccess) return e;
  return run_eval<PhysTTH>(a, st);
}
size_t cache_size_tth() { return cache_bytes<PhysTTH>(); }

}  // namespace mem

#include "mem_batch.cuh"

namespace mem {
// adaptive rounds; prepare_tth() must have run on this device (outside any capture)
cudaError_t launch_batch_tth(const BatchArgs& b, cudaStream_t st) {
  return run_batch<PhysTTH, MINB_TH>(b, st);
}
}  // namespace mem
