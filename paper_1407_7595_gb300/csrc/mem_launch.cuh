// Generic host launchers for one process's kernels (included by the
// per-process translation units).
#pragma once
#include "mem_internal.h"
#include "mem_kernels.cuh"

namespace mem {

// MINB: resident CTAs per SM the adaptation kernel is built for; MINB_MAIN: the
// same for the frozen-grid kernel (its register budget is 65536 / (256 MINB_MAIN)).
template <class PH, int PPT, int MINB, int MINB_MAIN = MINB>
cudaError_t run_integrate(const IntegrateArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(AdaptSmem<PH>);
  // set on every call: the attribute belongs to the current device's context
  cudaError_t ea = cudaFuncSetAttribute(k_adapt<PH, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
  if (ea != cudaSuccess) return ea;
  if (a.phase_events) cudaEventRecord(a.phase_events[0], st);
  // with n_iters == 0 the starting grid is frozen as given
  k_adapt<PH, MINB><<<(unsigned)a.n_items, THREADS, smem, st>>>(
      a.recs, a.P, a.T, a.n_items, philox_key(a.seed), a.event_id_base, a.n_iters, a.n_adapt, a.alpha,
      a.grid_in, a.grid32, reinterpret_cast<typename PH::Cache*>(a.caches));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.phase_events) cudaEventRecord(a.phase_events[1], st);
  const uint64_t blocks = (uint64_t)a.n_items * a.chunks_per_item;
  if (a.strat_k) {
    k_main_strat<PH, MINB_MAIN><<<(unsigned)blocks, THREADS, 0, st>>>(
        a.recs, a.P, a.T, a.n_items, a.chunks_per_item, philox_key(a.seed), a.event_id_base,
        a.idx0, a.strat_ns, a.strat_cubes, a.strat_k, a.cubes_per_thread, a.grid32,
        reinterpret_cast<const typename PH::Cache*>(a.caches), a.slots);
    return cudaGetLastError();
  }
  k_main<PH, PPT, MINB_MAIN><<<(unsigned)blocks, THREADS, 0, st>>>(
      a.recs, a.P, a.T, a.n_items, a.chunks_per_item, philox_key(a.seed), a.event_id_base, a.idx0, a.n_main,
      a.grid32, reinterpret_cast<const typename PH::Cache*>(a.caches), a.slots);
  return cudaGetLastError();
}

template <class PH>
size_t cache_bytes() {
  return sizeof(typename PH::Cache);
}

template <class PH>
cudaError_t run_eval(const EvalArgs& a, cudaStream_t st) {
  const unsigned blocks = (unsigned)((a.n + THREADS - 1) / THREADS);
  k_eval<PH><<<blocks, THREADS, 0, st>>>(a.rec, a.perm, a.P, a.T, philox_key(a.seed), a.event_id, a.point0,
                                         a.n, a.gb, a.w_out);
  return cudaGetLastError();
}

}  // namespace mem
