// Kernel instantiations for the semileptonic ttbar process.
#include "mem_launch.cuh"

namespace mem {

cudaError_t launch_integrate_tt(const IntegrateArgs&, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_eval_tt(const EvalArgs&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace mem

namespace mem {
size_t cache_size_tt() { return 16; }
}  // namespace mem
