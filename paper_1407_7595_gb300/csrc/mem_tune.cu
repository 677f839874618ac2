// Autotuner of the batched adaptive schedule (mem_plan) of one process: times
// a fixed list of candidate plans on calibration events through
// mem_integrate_batch and keeps the one with the most converged events per
// second. Host code only; the timed work is the library's own kernels.
#include <cuda_runtime.h>

#include <cfloat>
#include <string>
#include <vector>

#include "../../include/mem.h"
#include "mem_internal.h"

namespace {

mem_status tfail(mem_status s, const std::string& m) {
  mem::set_last_error(m.c_str());
  return s;
}

}  // namespace

extern "C" mem_status mem_autotune(const mem_events* events, const mem_process* process,
                                   const mem_tf_desc* tf, uint64_t seed, const mem_opts* opts,
                                   mem_plan* best, double* events_per_s, int32_t* n_tried,
                                   void* stream) {
  if (!events || events->magic != MAGIC_EVT || !process || process->magic != MAGIC_PROC || !tf ||
      !opts || !best)
    return tfail(MEM_ERR_INVALID_ARG, "invalid argument");
  if (!(opts->target_rel_err > 0.0)) return tfail(MEM_ERR_INVALID_ARG, "target_rel_err must be > 0");
  const int64_t n = events->n;
  if (n < 1) return tfail(MEM_ERR_INVALID_ARG, "no calibration events");
  cudaStream_t st = (cudaStream_t)stream;
  double *prob = nullptr, *err = nullptr;
  uint64_t* used = nullptr;
  int32_t* status = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaMalloc(&prob, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&err, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&used, n * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&status, n * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  std::vector<int32_t> h_status(n);
  int tried = 0;
  mem_status ms = e == cudaSuccess ? MEM_OK : MEM_ERR_CUDA;

  // converged events per second of one plan (0 if the plan does not fit the cap)
  auto rate_of = [&](const mem_plan& pl, double* rate) -> mem_status {
    *rate = 0.0;
    mem_opts o = *opts;
    o.plans = &pl;
    o.phase_events = nullptr;
    const mem_events* ev[1] = {events};
    const mem_process* pr[1] = {process};
    const mem_tf_desc* tfs[1] = {tf};
    mem_status s = mem_integrate_batch(1, ev, pr, tfs, seed, &o, prob, err, used, status, stream);
    if (s == MEM_ERR_INVALID_ARG) return MEM_OK;  // budget does not fit: not a candidate
    if (s != MEM_OK) return s;
    ++tried;
    float best_ms = FLT_MAX;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(t0, st);
      s = mem_integrate_batch(1, ev, pr, tfs, seed + 1 + rep, &o, prob, err, used, status, stream);
      if (s != MEM_OK) return s;
      cudaEventRecord(t1, st);
      if (cudaEventSynchronize(t1) != cudaSuccess) return MEM_ERR_CUDA;
      float m = 0.f;
      cudaEventElapsedTime(&m, t0, t1);
      best_ms = m < best_ms ? m : best_ms;
    }
    if (cudaMemcpy(h_status.data(), status, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return MEM_ERR_CUDA;
    int64_t conv = 0;
    for (int64_t i = 0; i < n; ++i) conv += h_status[i] == MEM_OK;
    *rate = (double)conv / (best_ms * 1e-3);
    return MEM_OK;
  };

  mem_plan top{};
  double top_rate = -1.0;
  auto consider = [&](const mem_plan& pl) {
    if (ms != MEM_OK) return;
    double r = 0.0;
    ms = rate_of(pl, &r);
    if (ms == MEM_OK && r > top_rate) {
      top_rate = r;
      top = pl;
    }
  };
  // stage 1: adaptation plan (iterations x points per item)
  const uint64_t min0 = opts->min_points ? opts->min_points : (uint64_t)1 << 14;
  const int stage1[][2] = {{2, 2048}, {3, 2048}, {2, 4096}, {3, 4096}, {4, 4096},
                           {5, 4096}, {2, 8192}, {3, 8192}, {5, 8192}};
  for (const auto& c : stage1) {
    mem_plan pl{};
    pl.n_adapt_iters = c[0];
    pl.adapt_points = (uint64_t)c[1];
    pl.min_points = min0;
    pl.tiles_per_cta = 4;
    consider(pl);
  }
  // stage 2: first-round size, then tiles per CTA, around the best plan
  if (ms == MEM_OK && top_rate > 0.0) {
    const mem_plan base = top;
    for (uint64_t m : {min0 / 2, min0 * 2}) {
      mem_plan pl = base;
      pl.min_points = m;
      consider(pl);
    }
    const mem_plan base2 = top;
    for (int t : {2, 8}) {
      mem_plan pl = base2;
      pl.tiles_per_cta = t;
      consider(pl);
    }
  }
  cudaFree(prob);
  cudaFree(err);
  cudaFree(used);
  cudaFree(status);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (ms != MEM_OK) return ms == MEM_ERR_CUDA ? tfail(ms, "mem_autotune: CUDA error") : ms;
  if (top_rate <= 0.0) return tfail(MEM_NOT_CONVERGED, "mem_autotune: no plan converged any event");
  *best = top;
  if (events_per_s) *events_per_s = top_rate;
  if (n_tried) *n_tried = tried;
  return MEM_OK;
}
