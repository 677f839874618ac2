// Kernel instantiations for the semileptonic ttbar process.
#include "mem_launch.cuh"
#include "mem_ttbar.cuh"

namespace mem {

constexpr int PPT_TT = 8;
constexpr int MINB_TT = 2;       // adaptation and round kernels: <= 128 registers, no spills
constexpr int MINB_TT_MAIN = 3;  // frozen-grid kernel: <= 80 registers (20 bytes of spill), 24 warps/SM

cudaError_t launch_integrate_tt(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysTT, PPT_TT, MINB_TT, MINB_TT_MAIN>(a, st);
}
cudaError_t launch_eval_tt(const EvalArgs& a, cudaStream_t st) { return run_eval<PhysTT>(a, st); }
size_t cache_size_tt() { return cache_bytes<PhysTT>(); }

}  // namespace mem

#include "mem_batch.cuh"

namespace mem {
cudaError_t launch_batch_tt(const BatchArgs& b, cudaStream_t st) { return run_batch<PhysTT, MINB_TT>(b, st); }
}  // namespace mem
