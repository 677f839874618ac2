// Learned sampler in the ttbar integral: the training-set generator, the
// adaptive-budget integral with VEGAS as fallback and judge, and per-point
// evaluation for parity checks (C entry points).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mem.h"
#include "mem_flow_int.cuh"
#include "mem_internal.h"

namespace mem {

constexpr int MINB_FLOW = 2;  // two 112 KB sampling CTAs per SM, <= 128 registers

// Per event, after the flow pilot: an item is judged by VEGAS when its variance
// per point exceeds tau I^2 / nperm (I = sum of the item means of the event),
// or when I is not positive. Items of events with an invalid record are not.
__global__ void k_flow_screen(int64_t n_events, int nperm, double tau,
                              const ItemAcc* __restrict__ acc, uint8_t* __restrict__ judge) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_events) return;
  double I = 0.0;
  bool invalid = false;
  for (int p = 0; p < nperm; ++p) {
    const ItemAcc A = acc[e * nperm + p];
    I += (A.s1 + A.c1) / (double)A.n;
    invalid |= A.pad != 0;
  }
  for (int p = 0; p < nperm; ++p) {
    const ItemAcc A = acc[e * nperm + p];
    const double N = (double)A.n, m = (A.s1 + A.c1) / N;
    const double var = (A.s2 + A.c2) / N - m * m;
    const bool j = !invalid && (!(I > 0.0) || var > tau * I * I / nperm);
    judge[e * nperm + p] = j ? 1 : 0;
  }
}

// Judged items: VEGAS (moments of its last adaptation iteration) against the
// flow pilot. sampler: 0 flow, 1 flow kept, 2 VEGAS.
__global__ void k_flow_judge(int64_t n_items, uint32_t n_adapt, double cost,
                             const uint8_t* __restrict__ judge, const Slot* __restrict__ mom,
                             const ItemAcc* __restrict__ acc, uint8_t* __restrict__ sampler) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  if (!judge[i]) {
    sampler[i] = 0;
    return;
  }
  const ItemAcc A = acc[i];
  const double N = (double)A.n, mf = (A.s1 + A.c1) / N;
  const double var_f = (A.s2 + A.c2) / N - mf * mf;
  const Slot V = mom[i];
  const double M = (double)n_adapt, mv = (V.s1 + V.c1) / M;
  const double var_v = (V.s2 + V.c2) / M - mv * mv;
  sampler[i] = var_f * cost <= var_v ? 1 : 2;
}

// sampler codes -> the sampler index of the round lists (0 flow, 1 VEGAS)
__global__ void k_flow_route(int64_t n_items, const uint8_t* __restrict__ sampler,
                             uint8_t* __restrict__ route) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_items) route[i] = sampler[i] == 2 ? 1 : 0;
}

size_t flow_samp_smem() { return sizeof(FlowSampSmem<PhysTT>); }

// Dynamic shared memory of a kernel, with the largest carveout preferred so that
// two 112 KB sampling CTAs fit on one SM (the occupancy query and the launch
// otherwise assume the default carveout and place one).
template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

}  // namespace mem

using namespace mem;

namespace {

mem_status ffail(mem_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t up(size_t b) { return (b + 255) & ~(size_t)255; }

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

mem_status check_tt(const mem_events* ev, const mem_process* pr, const mem_tf_desc* tf) {
  if (!ev || ev->magic != MAGIC_EVT || !pr || pr->magic != MAGIC_PROC || !tf)
    return ffail(MEM_ERR_INVALID_ARG, "invalid handle or tf");
  if (pr->desc.kind != PROC_TTBAR || ev->kind != PROC_TTBAR)
    return ffail(MEM_ERR_INVALID_ARG, "the learned sampler is built for the ttbar process");
  if (!(tf->met_sigma > 0 && tf->met_box_k > 0))
    return ffail(MEM_ERR_INVALID_ARG, "MET TF parameters invalid");
  return MEM_OK;
}

mem_status cuda_fail(const char* where, cudaError_t e) {
  return ffail(e == cudaErrorMemoryAllocation ? MEM_ERR_OOM : MEM_ERR_CUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

mem_status mem_flow_samples(const mem_events* events, const mem_process* process,
                            const mem_tf_desc* tf, uint64_t seed, const mem_opts* opts,
                            int32_t per_event, float* ys, float* ws, float* cs, float* log_jv,
                            void* stream) {
  mem_status s = check_tt(events, process, tf);
  if (s != MEM_OK) return s;
  if (!ys || !ws || !cs) return ffail(MEM_ERR_INVALID_ARG, "NULL output");
  if (per_event != 0 && per_event != 1) return ffail(MEM_ERR_INVALID_ARG, "per_event must be 0 or 1");
  const int iters = opts ? opts->n_adapt_iters : 5;
  const uint64_t n_adapt = opts && opts->adapt_points ? opts->adapt_points : 8192;
  const double alpha = opts && opts->alpha > 0 ? opts->alpha : 1.5;
  if (iters < 0 || iters > 64 || n_adapt > (1u << 24))
    return ffail(MEM_ERR_INVALID_ARG, "adaptation plan out of range");
  const int64_t n_items = events->n * PhysTT::NPERM;
  if (n_items < 1) return MEM_OK;
  const uint64_t eid0 = opts ? opts->event_id_base : 0;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t gb_bytes = up((size_t)n_items * PhysTT::D * NG * sizeof(GridBin));
  const size_t c_bytes = up((size_t)n_items * sizeof(TTCache));
  const size_t total = gb_bytes + c_bytes + up((size_t)n_items * sizeof(double));
  unsigned char* w = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&w, total, st);
  if (e != cudaSuccess) return cuda_fail("mem_flow_samples", e);
  GridBin* grid32 = reinterpret_cast<GridBin*>(w);
  TTCache* caches = reinterpret_cast<TTCache*>(w + gb_bytes);
  double* tot = reinterpret_cast<double*>(w + gb_bytes + c_bytes);
  const ProcConst P = process->pc;
  const TFConst T = make_tf_const_from(tf);
  const size_t smem = sizeof(AdaptSmem<PhysTT>);
  e = set_smem(k_adapt<PhysTT, MINB_FLOW>, smem);
  if (e == cudaSuccess) {
    k_adapt<PhysTT, MINB_FLOW><<<(unsigned)n_items, THREADS, smem, st>>>(
        events->d_recs, P, T, n_items, philox_key(seed), eid0, iters, (uint32_t)n_adapt, alpha, nullptr,
        grid32, caches);
    k_flow_samples<PhysTT><<<(unsigned)n_items, FTS, 0, st>>>(
        events->d_recs, P, n_items, philox_key(seed), eid0, (uint32_t)(iters * n_adapt), grid32, caches, ys,
        ws, cs, tot, log_jv);
    k_flow_normalise<<<(unsigned)n_items, FTS, 0, st>>>(n_items, PhysTT::NPERM, per_event, tot, ws);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(w, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("mem_flow_samples", e);
  return MEM_OK;
}

mem_status mem_set_tc_wait_limit(uint32_t polls) {
  cudaError_t e = cudaMemcpyToSymbol(mem::c_tc_wait_limit, &polls, sizeof(polls));
  if (e == cudaSuccess) e = mem::set_train_wait_limit(polls);
  if (e != cudaSuccess) return cuda_fail("mem_set_tc_wait_limit", e);
  return MEM_OK;
}

mem_status mem_flow_eval_points(const mem_process* process, const mem_tf_desc* tf,
                                const mem_flow* flow, const float* record, int32_t perm,
                                uint64_t seed, uint32_t event_id, uint32_t point0, int64_t n,
                                float* z, float* logj, double* w, void* stream) {
  if (!process || process->magic != MAGIC_PROC || process->desc.kind != PROC_TTBAR || !tf ||
      !flow || flow->magic != MAGIC_FLOW || !record || !z || !logj || !w || perm < 0 ||
      perm >= PhysTT::NPERM || n < 1 || n > ((int64_t)1 << 30))
    return ffail(MEM_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t smem = flow_samp_smem();
  int* d_err = nullptr;
  int h_err = 0;
  cudaError_t e = set_smem(k_flow_points<PhysTT, MINB_FLOW>, smem);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_err, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)((n + FCH - 1) / FCH);
    k_flow_points<PhysTT, MINB_FLOW><<<blocks, THREADS, smem, st>>>(
        record, perm, process->pc, make_tf_const_from(tf), philox_key(seed), event_id, point0, (uint32_t)n,
        flow->W, flow->B, z, logj, w, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (d_err) cudaFreeAsync(d_err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("mem_flow_eval_points", e);
  if (h_err) return ffail(MEM_ERR_TIMEOUT, "mem_flow_eval_points: a tensor-core wait gave up");
  return MEM_OK;
}

mem_status mem_integrate_flow(const mem_events* events, const mem_process* process,
                              const mem_tf_desc* tf, const mem_flow* flow, uint64_t seed,
                              const mem_opts* opts, double* prob, double* err, uint64_t* n_used,
                              int32_t* ev_status, uint8_t* item_sampler, void* stream) {
  mem_status s = check_tt(events, process, tf);
  if (s != MEM_OK) return s;
  if (!flow || flow->magic != MAGIC_FLOW || !opts || !prob || !err)
    return ffail(MEM_ERR_INVALID_ARG, "invalid argument");
  if (!(opts->target_rel_err > 0.0)) return ffail(MEM_ERR_INVALID_ARG, "target_rel_err must be > 0");
  if (opts->flow_guided != 0 && opts->flow_guided != 1)
    return ffail(MEM_ERR_INVALID_ARG, "flow_guided must be 0 or 1");
  if (opts->grid_in) return ffail(MEM_ERR_INVALID_ARG, "grid_in is not supported with the flow");
  const bool guided = opts->flow_guided == 1;
  constexpr int NP = PhysTT::NPERM;
  const int iters = opts->n_adapt_iters ? opts->n_adapt_iters : 5;
  const uint64_t n_adapt = opts->adapt_points ? opts->adapt_points : 8192;
  if (iters < 1 || iters > 64 || n_adapt > (1u << 24))
    return ffail(MEM_ERR_INVALID_ARG, "adaptation plan out of range");
  const double alpha = opts->alpha > 0 ? opts->alpha : 1.5;
  const double tau = opts->flow_screen != 0.0 ? opts->flow_screen : 1.0;
  const double cost = opts->flow_cost > 0.0 ? opts->flow_cost : 1.0;
  const uint64_t cap_ev = opts->max_points ? opts->max_points : (uint64_t)1 << 24;
  const uint64_t min_ev = opts->min_points ? opts->min_points : (uint64_t)1 << 14;
  const uint64_t cap_item = cap_ev / NP, adapt = (uint64_t)iters * n_adapt;
  uint64_t pts0 = (min_ev / NP + FROWS - 1) / FROWS * FROWS;
  pts0 = pts0 < FROWS ? FROWS : pts0;
  if (cap_item < adapt + pts0)
    return ffail(MEM_ERR_INVALID_ARG, "max_points too small for the pilot and the VEGAS judge");
  int rounds = 1;
  while (adapt + pts0 * ((((uint64_t)1) << (rounds + 1)) - 1) <= cap_item && rounds < 24) ++rounds;
  if (adapt + pts0 * ((((uint64_t)1) << rounds) - 1) > ((uint64_t)1 << 32))
    return ffail(MEM_ERR_INVALID_ARG, "point budget above 2^32 per item");
  const int64_t n_ev = events->n, n_items = n_ev * NP;
  if (n_ev < 1) return MEM_OK;

  // workspace
  const int sms = sm_count();
  int occ_f = 0, occ_v = 0, occ_a = 0;
  const size_t smem_f = flow_samp_smem(), smem_a = sizeof(AdaptSmem<PhysTT>);
  cudaError_t e = set_smem(k_flow_round_sample<PhysTT, MINB_FLOW, false>, smem_f);
  if (e == cudaSuccess) e = set_smem(k_flow_round_sample<PhysTT, MINB_FLOW, true>, smem_f);
  if (e == cudaSuccess) e = set_smem(k_adapt_list<PhysTT, MINB_FLOW>, smem_a);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_f, k_flow_round_sample<PhysTT, MINB_FLOW, false>, THREADS, smem_f);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_v, k_round_sample<PhysTT, MINB_FLOW>,
                                                      THREADS, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, k_adapt_list<PhysTT, MINB_FLOW>,
                                                      THREADS, smem_a);
  if (e != cudaSuccess) return cuda_fail("mem_integrate_flow", e);
  // the sampling kernel is built for MINB_FLOW CTAs per SM (launch bounds and
  // shared memory); the occupancy query can under-report it for kernels that
  // use tensor memory, and surplus CTAs of the persistent loop only queue
  occ_f = occ_f > MINB_FLOW ? occ_f : MINB_FLOW;
  const int ctas_f = occ_f * sms, ctas_v = (occ_v > 0 ? occ_v : 1) * sms;
  const int ctas_a = (occ_a > 0 ? occ_a : 1) * sms;
  const int tt_f = 2 * ctas_f, tt_v = 4 * ctas_v;
  const size_t slots_f = (size_t)n_items + tt_f + 1024, slots_v = (size_t)n_items + tt_v + 1024;
  size_t total = 0;
  const size_t o_grid = total; total += up((size_t)n_items * PhysTT::D * NG * sizeof(GridBin));
  const size_t o_cache = total; total += up((size_t)n_items * sizeof(TTCache));
  const size_t o_feat = total; total += up((size_t)n_items * FC * sizeof(float));
  const size_t o_acc = total; total += up((size_t)n_items * sizeof(ItemAcc));
  const size_t o_mom = total; total += up((size_t)n_items * sizeof(Slot));
  const size_t o_actf = total; total += up((size_t)n_items * sizeof(int32_t));
  const size_t o_actv = total; total += up((size_t)n_items * sizeof(int32_t));
  const size_t o_flags = total; total += up((size_t)n_items);
  const size_t o_judge = total; total += up((size_t)n_items);
  const size_t o_samp = total; total += up((size_t)n_items);
  const size_t o_route = total; total += up((size_t)n_items);
  const size_t o_ctl = total; total += up(2 * sizeof(RoundCtl));
  const size_t o_slf = total; total += up(slots_f * sizeof(Slot));
  const size_t o_slv = total; total += up(slots_v * sizeof(Slot));
  const size_t o_state = total; total += up((size_t)n_ev * sizeof(int32_t));
  const size_t o_eflag = total; total += up(sizeof(int));
  const size_t o_hist = total;
  if (guided) total += up((size_t)n_items * PhysTT::D * NG * sizeof(float));
  const bool dev_out = dev_ptr(prob);
  const size_t o_out = total;
  if (!dev_out) total += 4 * up((size_t)n_ev * 8);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = nullptr;
  e = cudaMallocAsync((void**)&w, total, st);
  if (e != cudaSuccess) return cuda_fail("mem_integrate_flow: workspace", e);
  GridBin* grid32 = reinterpret_cast<GridBin*>(w + o_grid);
  TTCache* caches = reinterpret_cast<TTCache*>(w + o_cache);
  float* feats = reinterpret_cast<float*>(w + o_feat);
  ItemAcc* acc = reinterpret_cast<ItemAcc*>(w + o_acc);
  Slot* mom = reinterpret_cast<Slot*>(w + o_mom);
  int32_t* act_f = reinterpret_cast<int32_t*>(w + o_actf);
  int32_t* act_v = reinterpret_cast<int32_t*>(w + o_actv);
  uint8_t* flags = w + o_flags;
  uint8_t* judge = w + o_judge;
  uint8_t* sampler = w + o_samp;
  uint8_t* route = w + o_route;
  RoundCtl* ctl_f = reinterpret_cast<RoundCtl*>(w + o_ctl);
  RoundCtl* ctl_v = ctl_f + 1;
  Slot* sl_f = reinterpret_cast<Slot*>(w + o_slf);
  Slot* sl_v = reinterpret_cast<Slot*>(w + o_slv);
  int32_t* ev_state = reinterpret_cast<int32_t*>(w + o_state);
  float* hist = guided ? reinterpret_cast<float*>(w + o_hist) : nullptr;
  int* d_err = reinterpret_cast<int*>(w + o_eflag);
  int h_err = 0;
  double* o_prob = dev_out ? prob : reinterpret_cast<double*>(w + o_out);
  double* o_err = dev_out ? err : reinterpret_cast<double*>(w + o_out + up((size_t)n_ev * 8));
  uint64_t* o_used = dev_out ? n_used : reinterpret_cast<uint64_t*>(w + o_out + 2 * up((size_t)n_ev * 8));
  int32_t* o_st = dev_out ? ev_status : reinterpret_cast<int32_t*>(w + o_out + 3 * up((size_t)n_ev * 8));

  const float* recs = events->d_recs;
  const ProcConst P = process->pc;
  const TFConst T = make_tf_const_from(tf);
  const uint64_t eid0 = opts->event_id_base;
  const PhiloxKey key = philox_key(seed);
  const unsigned gi = (unsigned)((n_items + 255) / 256), ge = (unsigned)((n_ev + 127) / 128);

  // the whole schedule is captured into one CUDA graph on a private stream
  cudaStream_t cs = nullptr;
  cudaEvent_t join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(join, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    k_flow_setup<PhysTT><<<gi, 256, 0, cs>>>(recs, P, T, n_items, caches, feats);
    cudaMemsetAsync(d_err, 0, sizeof(int), cs);
    cudaMemsetAsync(acc, 0, (size_t)n_items * sizeof(ItemAcc), cs);
    cudaMemsetAsync(ev_state, 0, (size_t)n_ev * sizeof(int32_t), cs);
    cudaMemsetAsync(flags, 1, (size_t)n_items, cs);
    // round 0: flow pilot on every item
    k_round_compact<<<1, 1024, 0, cs>>>(n_items, flags, act_f, ctl_f, tt_f, nullptr, 0);
    if (guided) {
      cudaMemsetAsync(hist, 0, (size_t)n_items * PhysTT::D * NG * sizeof(float), cs);
      k_flow_round_sample<PhysTT, MINB_FLOW, true><<<ctas_f, THREADS, smem_f, cs>>>(
          recs, P, key, eid0, act_f, ctl_f, 0u, (uint32_t)pts0, flow->W, flow->B, caches, feats,
          sl_f, hist, d_err);
    } else {
      k_flow_round_sample<PhysTT, MINB_FLOW, false><<<ctas_f, THREADS, smem_f, cs>>>(
          recs, P, key, eid0, act_f, ctl_f, 0u, (uint32_t)pts0, flow->W, flow->B, caches, feats,
          sl_f, nullptr, d_err);
    }
    k_round_reduce<<<gi, 256, 0, cs>>>(act_f, ctl_f, (uint32_t)pts0, sl_f, acc);
    // screen, VEGAS judge on the flagged items, sampler per item
    k_flow_screen<<<ge, 128, 0, cs>>>(n_ev, NP, tau, acc, judge);
    k_round_compact<<<1, 1024, 0, cs>>>(n_items, judge, act_v, ctl_v, tt_v, nullptr, 0);
    k_adapt_list<PhysTT, MINB_FLOW><<<ctas_a, THREADS, smem_a, cs>>>(
        recs, P, T, act_v, &ctl_v->n_active, key, eid0, iters, (uint32_t)n_adapt, alpha, grid32,
        caches, mom, hist);
    k_flow_judge<<<gi, 256, 0, cs>>>(n_items, (uint32_t)n_adapt, cost, judge, mom, acc, sampler);
    k_flow_route<<<gi, 256, 0, cs>>>(n_items, sampler, route);
    k_round_check<<<ge, 128, 0, cs>>>(n_ev, NP, opts->target_rel_err, P.prefactor, rounds == 1,
                                      pts0 * 4, acc, ev_state, flags);
    uint64_t pts = pts0, idx_f = pts0;
    for (int r = 1; r < rounds; ++r) {
      pts *= 2;
      k_round_compact<<<1, 1024, 0, cs>>>(n_items, flags, act_f, ctl_f, tt_f, route, 0);
      k_round_compact<<<1, 1024, 0, cs>>>(n_items, flags, act_v, ctl_v, tt_v, route, 1);
      k_flow_round_sample<PhysTT, MINB_FLOW, false><<<ctas_f, THREADS, smem_f, cs>>>(
          recs, P, key, eid0, act_f, ctl_f, (uint32_t)idx_f, (uint32_t)pts, flow->W, flow->B,
          caches, feats, sl_f, nullptr, d_err);
      k_round_sample<PhysTT, MINB_FLOW><<<ctas_v, THREADS, 0, cs>>>(
          recs, P, key, eid0, act_v, ctl_v, (uint32_t)(adapt + idx_f), (uint32_t)pts, grid32,
          caches, sl_v);
      k_round_reduce<<<gi, 256, 0, cs>>>(act_f, ctl_f, (uint32_t)pts, sl_f, acc);
      k_round_reduce<<<gi, 256, 0, cs>>>(act_v, ctl_v, (uint32_t)pts, sl_v, acc);
      k_round_check<<<ge, 128, 0, cs>>>(n_ev, NP, opts->target_rel_err, P.prefactor,
                                        r == rounds - 1, pts0 * 4, acc, ev_state, flags);
      idx_f += pts;
    }
    k_batch_final<<<ge, 128, 0, cs>>>(n_ev, NP, P.prefactor, adapt, acc, ev_state, judge, o_prob,
                                      o_err, o_used, o_st);
    cudaError_t ce = cudaGetLastError();
    e = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ce;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
  if (e == cudaSuccess) e = cudaEventRecord(join, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join, 0);
  if (e == cudaSuccess && !dev_out) {
    e = cudaMemcpyAsync(prob, o_prob, n_ev * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err, o_err, n_ev * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n_used)
      e = cudaMemcpyAsync(n_used, o_used, n_ev * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ev_status)
      e = cudaMemcpyAsync(ev_status, o_st, n_ev * 4, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && item_sampler)
    e = cudaMemcpyAsync(item_sampler, sampler, (size_t)n_items, dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaFreeAsync(w, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (join) cudaEventDestroy(join);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail("mem_integrate_flow", e);
  if (h_err) return ffail(MEM_ERR_TIMEOUT, "mem_integrate_flow: a tensor-core wait gave up");
  return MEM_OK;
}

}  // extern "C"
