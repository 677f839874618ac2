// Kernel instantiations for the semileptonic ttbar process (parametric PDFs; the
// tabulated-PDF builds are in mem_launch_grid.cu).
#include "mem_launch.cuh"
#include "mem_launch_config.h"
#include "mem_ttbar.cuh"

namespace mem {

cudaError_t launch_integrate_tt(const IntegrateArgs& a, cudaStream_t st) {
  if (a.P.pdf_grid) return launch_integrate_tt_grid(a, st);
  return run_integrate<PhysTT_<PDF_PARAM>, PPT_TT, MINB_TT, MINB_TT_MAIN>(a, st);
}
cudaError_t launch_eval_tt(const EvalArgs& a, cudaStream_t st) { return run_eval<PhysTT>(a, st); }
size_t cache_size_tt() { return cache_bytes<PhysTT>(); }

}  // namespace mem

#include "mem_batch.cuh"

namespace mem {
cudaError_t launch_batch_tt(const BatchArgs& b, cudaStream_t st) {
  if (b.base.P.pdf_grid) return launch_batch_tt_grid(b, st);
  return run_batch<PhysTT_<PDF_PARAM>, MINB_TT>(b, st);
}
}  // namespace mem
