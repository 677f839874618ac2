// Kernel instantiations of the three processes with tabulated PDFs (Sec. 3:
// per-flavour (x, Q) grids, bilinear interpolation), launched when a table is
// attached to the process. A separate translation unit: it compiles in parallel
// with the parametric builds.
#include "mem_launch.cuh"
#include "mem_launch_config.h"
#include "mem_ttbar.cuh"
#include "mem_batch.cuh"

namespace mem {

cudaError_t launch_integrate_dy_grid(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysDY_<PDF_GRID>, PPT_DY, 1>(a, st);
}
cudaError_t launch_integrate_w_grid(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysW_<PDF_GRID>, PPT_W, MINB_W, MINB_W_MAIN>(a, st);
}
cudaError_t launch_integrate_tt_grid(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysTT_<PDF_GRID>, PPT_TT, MINB_TT, MINB_TT_MAIN>(a, st);
}
cudaError_t launch_batch_dy_grid(const BatchArgs& b, cudaStream_t st) {
  return run_batch<PhysDY_<PDF_GRID>, 1>(b, st);
}
cudaError_t launch_batch_w_grid(const BatchArgs& b, cudaStream_t st) {
  return run_batch<PhysW_<PDF_GRID>, MINB_W>(b, st);
}
cudaError_t launch_batch_tt_grid(const BatchArgs& b, cudaStream_t st) {
  return run_batch<PhysTT_<PDF_GRID>, MINB_TT>(b, st);
}

}  // namespace mem
