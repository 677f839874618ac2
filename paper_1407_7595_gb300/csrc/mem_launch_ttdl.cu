// Kernel instantiations for the dilepton ttbar process. One build serves the
// parametric and the tabulated PDFs (chosen per call): the FP64 neutrino solution
// dominates this integrand, not the PDF lookup.
#include "mem_launch.cuh"
#include "mem_launch_config.h"
#include "mem_ttdl.cuh"

namespace mem {

cudaError_t launch_integrate_ttdl(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysTTDL, PPT_DL, MINB_DL, MINB_DL_MAIN>(a, st);
}
cudaError_t launch_eval_ttdl(const EvalArgs& a, cudaStream_t st) { return run_eval<PhysTTDL>(a, st); }
size_t cache_size_ttdl() { return cache_bytes<PhysTTDL>(); }

}  // namespace mem

#include "mem_batch.cuh"

namespace mem {
cudaError_t launch_batch_ttdl(const BatchArgs& b, cudaStream_t st) {
  return run_batch<PhysTTDL, MINB_DL>(b, st);
}
}  // namespace mem
