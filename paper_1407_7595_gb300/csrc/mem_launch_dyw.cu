// Kernel instantiations for the Drell-Yan and W processes.
#include "mem_launch.cuh"

namespace mem {

constexpr int PPT_DY = 16;
constexpr int PPT_W = 32;
constexpr int MINB_W = 5;       // adaptation and round kernels: 5 CTAs of 256 threads per SM (<= 51 registers)
constexpr int MINB_W_MAIN = 6;  // frozen-grid kernel: 6 CTAs per SM (<= 42 registers, 4 bytes of spill)

cudaError_t launch_integrate_dy(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysDY, PPT_DY, 1>(a, st);
}
cudaError_t launch_integrate_w(const IntegrateArgs& a, cudaStream_t st) {
  return run_integrate<PhysW, PPT_W, MINB_W, MINB_W_MAIN>(a, st);
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
cudaError_t launch_batch_dy(const BatchArgs& b, cudaStream_t st) { return run_batch<PhysDY, 1>(b, st); }
cudaError_t launch_batch_w(const BatchArgs& b, cudaStream_t st) { return run_batch<PhysW, MINB_W>(b, st); }
}  // namespace mem
