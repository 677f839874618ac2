// Kernel instantiations for the Drell-Yan and W processes (parametric PDFs; the
// tabulated-PDF builds are in mem_launch_grid.cu).
#include "mem_launch.cuh"
#include "mem_launch_config.h"

namespace mem {

cudaError_t launch_integrate_dy(const IntegrateArgs& a, cudaStream_t st) {
  if (a.P.pdf_grid) return launch_integrate_dy_grid(a, st);
  return run_integrate<PhysDY_<PDF_PARAM>, PPT_DY, 1>(a, st);
}
cudaError_t launch_integrate_w(const IntegrateArgs& a, cudaStream_t st) {
  if (a.P.pdf_grid) return launch_integrate_w_grid(a, st);
  return run_integrate<PhysW_<PDF_PARAM>, PPT_W, MINB_W, MINB_W_MAIN>(a, st);
}
cudaError_t launch_eval_dy(const EvalArgs& a, cudaStream_t st) { return run_eval<PhysDY>(a, st); }
cudaError_t launch_eval_w(const EvalArgs& a, cudaStream_t st) { return run_eval<PhysW>(a, st); }

}  // namespace mem

namespace mem {
size_t cache_size_dy() { return cache_bytes<PhysDY>(); }
size_t cache_size_w() { return cache_bytes<PhysW>(); }
}  // namespace mem

#include "mem_batch.cuh"

namespace mem {
cudaError_t launch_batch_dy(const BatchArgs& b, cudaStream_t st) {
  if (b.base.P.pdf_grid) return launch_batch_dy_grid(b, st);
  return run_batch<PhysDY_<PDF_PARAM>, 1>(b, st);
}
cudaError_t launch_batch_w(const BatchArgs& b, cudaStream_t st) {
  if (b.base.P.pdf_grid) return launch_batch_w_grid(b, st);
  return run_batch<PhysW_<PDF_PARAM>, MINB_W>(b, st);
}
}  // namespace mem
