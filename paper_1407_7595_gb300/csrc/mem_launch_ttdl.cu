// Kernel instantiations for the dilepton ttbar process. One build serves the
// parametric and the tabulated PDFs (chosen per call): the FP64 neutrino solution
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
// FP64 inputs; solutions in GeV with their Jacobians, as the integrand uses them.
__global__ void k_dilep_solve(const double* __restrict__ in, int64_t n, int32_t* __restrict__ nsol,
                              double* __restrict__ out, double* __restrict__ jac) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* q = in + i * 22;
  const double iu = 1.0 / DL_UNIT, iu2 = iu * iu;
  double b[4], bb[4], lp[4], lm[4];
  for (int k = 0; k < 4; ++k) {
    b[k] = q[k] * iu;
    bb[k] = q[4 + k] * iu;
    lp[k] = q[8 + k] * iu;
    lm[k] = q[12 + k] * iu;
  }
  DLSystem S;
  double xr[4];
  const int nr = dl_system_met(b, bb, lp, lm, q[16] * iu, q[17] * iu, q[18] * iu2, q[19] * iu2,
                               q[20] * iu2, q[21] * iu2, S, xr);
  double seen[4][2];
  int ns = 0;
  for (int r = 0; r < nr; ++r) {
    double px, py;
    if (!dl_point(S, xr[r], px, py)) continue;
    bool dup = false;
    for (int k = 0; k < ns; ++k)
      dup = dup || fabs(seen[k][0] - px) + fabs(seen[k][1] - py) < 1e-9 * (1.0 + fabs(px) + fabs(py));
    if (dup) continue;
    seen[ns][0] = px;
    seen[ns][1] = py;
    double nu[4], nub[4];
    nu[1] = px;
    nu[2] = py;
    nu[3] = S.n1.z[0] + S.n1.z[1] * px + S.n1.z[2] * py;
    nu[0] = sqrt(px * px + py * py + nu[3] * nu[3]);
    nub[1] = S.mx - px;
    nub[2] = S.my - py;
    nub[3] = S.n2.z[0] + S.n2.z[1] * nub[1] + S.n2.z[2] * nub[2];
    nub[0] = sqrt(nub[1] * nub[1] + nub[2] * nub[2] + nub[3] * nub[3]);
    jac[i * 4 + ns] = dl_jacobian(b, bb, lp, lm, nu, nub);
    for (int k = 0; k < 4; ++k) {
      out[(i * 4 + ns) * 8 + k] = nu[k] * DL_UNIT;
      out[(i * 4 + ns) * 8 + 4 + k] = nub[k] * DL_UNIT;
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
