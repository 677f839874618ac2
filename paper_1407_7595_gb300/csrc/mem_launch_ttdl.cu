// Kernel instantiations for the dilepton ttbar process. One build serves the
// parametric and the tabulated PDFs (chosen per call): the neutrino solution
// dominates this integrand, not the PDF lookup.
#include <string>

#include "../../include/mem.h"
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

namespace mem {
namespace {

// One thread per system: the integrand's neutrino solution (dl_system_met, the
// real roots of the resultant, dl_point with its checks and de-duplication) on
// FP64 inputs rounded to double-float; solutions in GeV with their Jacobians, as
// the integrand uses them.
__global__ void k_dilep_solve(const double* __restrict__ in, int64_t n, int32_t* __restrict__ nsol,
                              double* __restrict__ out, double* __restrict__ jac) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* q = in + i * 22;
  const double u = (double)DL_UNIT, u2 = u * u;
  const DLMom b = dl_mom64(q), bb = dl_mom64(q + 4), lp = dl_mom64(q + 8), lm = dl_mom64(q + 12);
  DLSystem S;
  df xr[4];
  const int nr = dl_system_met(b, bb, lp, lm, df_from_double(q[16] / u), df_from_double(q[17] / u),
                               df_from_double(q[18] / u2), df_from_double(q[19] / u2),
                               df_from_double(q[20] / u2), df_from_double(q[21] / u2), S, xr);
  df seen[4][2];
  int ns = 0;
  for (int r = 0; r < nr; ++r) {
    df px, py;
    if (!dl_point(S, xr[r], px, py)) continue;
    bool dup = false;
    for (int k = 0; k < ns; ++k) dup = dup || dl_same(seen[k][0], seen[k][1], px, py);
    if (dup) continue;
    seen[ns][0] = px;
    seen[ns][1] = py;
    DLMom nu, nub;
    dl_neutrinos(S, px, py, nu, nub);
    const double det = to_double(dl_det(b, bb, lp, lm, nu, nub));
    jac[i * 4 + ns] = det > 0.0 ? 1.0 / (det * u2 * u2) : 0.0;
    for (int k = 0; k < 4; ++k) {
      out[(i * 4 + ns) * 8 + k] = to_double(nu.v[k]) * u;
      out[(i * 4 + ns) * 8 + 4 + k] = to_double(nub.v[k]) * u;
    }
    ++ns;
  }
  nsol[i] = ns;
}

}  // namespace
}  // namespace mem

extern "C" mem_status mem_dilep_solve(const double* in, int64_t n, int32_t* nsol, double* nu,
                                      double* jac) {
  if (!in || !nsol || !nu || !jac || n < 1 || n > ((int64_t)1 << 24)) {
    mem::set_last_error("mem_dilep_solve: invalid argument");
    return MEM_ERR_INVALID_ARG;
  }
  double *d_in = nullptr, *d_out = nullptr, *d_jac = nullptr;
  int32_t* d_n = nullptr;
  cudaError_t e = cudaMalloc(&d_in, (size_t)n * 22 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)n * 32 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_jac, (size_t)n * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_n, (size_t)n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, in, (size_t)n * 22 * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d_out, 0, (size_t)n * 32 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(d_jac, 0, (size_t)n * 4 * sizeof(double));
  if (e == cudaSuccess) {
    mem::k_dilep_solve<<<(unsigned)((n + 127) / 128), 128>>>(d_in, n, d_n, d_out, d_jac);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(nsol, d_n, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(nu, d_out, (size_t)n * 32 * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(jac, d_jac, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_in);
  cudaFree(d_out);
  cudaFree(d_jac);
  cudaFree(d_n);
  if (e != cudaSuccess) {
    const std::string m = std::string("mem_dilep_solve: ") + cudaGetErrorString(e);
    mem::set_last_error(m.c_str());
    return MEM_ERR_CUDA;
  }
  return MEM_OK;
}
