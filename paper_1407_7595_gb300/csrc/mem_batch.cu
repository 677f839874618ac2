// Batched adaptive-budget integration: round kernels that do not depend on the
// process, and the C entry point mem_integrate_batch (one CUDA graph per call).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mem.h"
#include "mem_batch.cuh"
#include "mem_internal.h"

namespace mem {

__global__ void k_round_reduce(const int32_t* __restrict__ active, const RoundCtl* __restrict__ ctl,
                               uint32_t pts_item, const Slot* __restrict__ slots,
                               ItemAcc* __restrict__ acc) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ctl->n_active) return;
  const int tpi = ctl->tiles_per_item;
  ItemAcc A = acc[active[a]];
  for (int k = 0; k < tpi; ++k) {
    const Slot q = slots[(int64_t)a * tpi + k];
    neu2(A.s1, A.c1, q.s1);
    neu2(A.s1, A.c1, q.c1);
    neu2(A.s2, A.c2, q.s2);
    neu2(A.s2, A.c2, q.c2);
    A.n_bad += q.n_bad & 0x7fffffffu;
    A.pad |= q.n_bad >> 31;  // invalid event record
  }
  A.n += pts_item;
  acc[active[a]] = A;
}

__global__ void k_round_check(int64_t n_events, int nperm, double target, double prefactor,
                              int last_round, uint64_t keep_n, const ItemAcc* __restrict__ acc,
                              int32_t* __restrict__ ev_state, uint8_t* __restrict__ flags) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_events) return;
  int32_t state = ev_state[e];
  double ms = 0, mc = 0, vs = 0, vc = 0;
  if (state == 0) {
    bool invalid = false;
    for (int p = 0; p < nperm; ++p) {
      const ItemAcc A = acc[e * nperm + p];
      const double N = (double)A.n;
      const double mean = (A.s1 + A.c1) / N;
      double var = ((A.s2 + A.c2) / N - mean * mean) / (N - 1.0);
      var = var > 0.0 ? var : 0.0;
      neu2(ms, mc, mean);
      neu2(vs, vc, var);
      invalid |= A.pad != 0;
    }
    const double prob = prefactor * (ms + mc) / nperm;
    const double err = prefactor * sqrt(vs + vc) / nperm;
    if (invalid) state = 3;
    else if (prob > 0.0 && err <= target * prob) state = 1;
    else if (last_round) state = 2;
    ev_state[e] = state;
  }
  // Items of an unconverged event keep sampling while their variance of the
  // mean exceeds a quarter of their equal share of the event's error budget
  // (target |sum of means|)^2 / nperm, or while they have no variance estimate
  // yet and fewer than keep_n points (support not found yet).
  const double tot = fabs(ms + mc);
  const double share = (target * tot) * (target * tot) / nperm;
  for (int p = 0; p < nperm; ++p) {
    uint8_t f = 0;
    if (state == 0) {
      const ItemAcc A = acc[e * nperm + p];
      const double N = (double)A.n;
      const double mean = (A.s1 + A.c1) / N;
      const double var = ((A.s2 + A.c2) / N - mean * mean) / (N - 1.0);
      f = (var > 0.25 * share || (!(var > 0.0) && A.n < keep_n) || !(tot > 0.0)) ? 1 : 0;
    }
    flags[e * nperm + p] = f;
  }
}

__global__ void k_round_compact(int64_t n_items, const uint8_t* __restrict__ flags,
                                int32_t* __restrict__ active, RoundCtl* __restrict__ ctl,
                                int target_tiles, const uint8_t* __restrict__ sel, int want) {
  // block-wide exclusive scan over chunks of blockDim items, in item order
  __shared__ int32_t wsum[32];
  __shared__ int32_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t off = 0; off < n_items; off += blockDim.x) {
    const int64_t i = off + threadIdx.x;
    const int f = (i < n_items) ? (flags[i] && (!sel || sel[i] == want)) : 0;
    int x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    const int incl = x + (warp > 0 ? wsum[warp - 1] : 0);
    if (f) active[base + incl - 1] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) base += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int n = base;
    ctl->n_active = n;
    int tpi = n > 0 ? (target_tiles + n - 1) / n : 1;
    tpi = tpi < 1 ? 1 : (tpi > 256 ? 256 : tpi);
    ctl->tiles_per_item = tpi;
  }
}

__global__ void k_batch_final(int64_t n_events, int nperm, double prefactor, uint64_t adapt_pts_item,
                              const ItemAcc* __restrict__ acc, const int32_t* __restrict__ ev_state,
                              const uint8_t* __restrict__ adapted, double* __restrict__ prob,
                              double* __restrict__ err, uint64_t* __restrict__ n_used,
                              int32_t* __restrict__ status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_events) return;
  double ms = 0, mc = 0, vs = 0, vc = 0;
  uint64_t n = 0;
  uint32_t bad = 0;
  for (int p = 0; p < nperm; ++p) {
    const ItemAcc A = acc[e * nperm + p];
    const double N = (double)A.n;
    const double mean = (A.s1 + A.c1) / N;
    double var = ((A.s2 + A.c2) / N - mean * mean) / (N - 1.0);
    var = var > 0.0 ? var : 0.0;
    neu2(ms, mc, mean);
    neu2(vs, vc, var);
    n += A.n + ((!adapted || adapted[e * nperm + p]) ? adapt_pts_item : 0);
    bad += A.n_bad;
  }
  prob[e] = prefactor * (ms + mc) / nperm;
  err[e] = prefactor * sqrt(vs + vc) / nperm;
  if (n_used) n_used[e] = n;
  const int32_t st = ev_state[e];
  if (status)
    status[e] = st == 3 ? MEM_ERR_INVALID_ARG
                        : (bad ? MEM_ERR_NONFINITE : (st == 1 ? MEM_OK : MEM_NOT_CONVERGED));
}

}  // namespace mem

namespace {

thread_local std::string g_batch_err;

mem_status bfail(mem_status s, const std::string& m) {
  mem::set_last_error(m.c_str());
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

}  // namespace

using namespace mem;

extern "C" mem_status mem_integrate_batch(int32_t n_groups, const mem_events* const* events,
                                          const mem_process* const* procs,
                                          const mem_tf_desc* const* tfs, uint64_t seed,
                                          const mem_opts* opts, double* prob, double* err,
                                          uint64_t* n_used, int32_t* ev_status, void* stream) {
  if (n_groups < 1 || n_groups > 16 || !events || !procs || !tfs || !opts || !prob || !err)
    return bfail(MEM_ERR_INVALID_ARG, "invalid argument");
  if (!(opts->target_rel_err > 0.0)) return bfail(MEM_ERR_INVALID_ARG, "target_rel_err must be > 0");
  if (opts->flow_guided != 0) return bfail(MEM_ERR_INVALID_ARG, "flow_guided must be 0");
  if (opts->strat_points != 0 || opts->reserved1 != 0)
    return bfail(MEM_ERR_INVALID_ARG, "strat_points must be 0 with adaptive budgets");
  const uint64_t cap_ev = opts->max_points ? opts->max_points : (uint64_t)1 << 24;
  const double alpha = opts->alpha > 0 ? opts->alpha : 1.5;
  if (opts->grid_in) return bfail(MEM_ERR_INVALID_ARG, "grid_in is not supported with adaptive budgets");

  struct Plan {
    BatchArgs b;
    size_t off_grid, off_cache, off_acc, off_act, off_flags, off_ctl, off_slots, off_state;
    int64_t ev_off;
  };
  std::vector<Plan> plans(n_groups);
  size_t total = 0;
  int64_t ev_total = 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int g = 0; g < n_groups; ++g) {
    const mem_events* ev = events[g];
    const mem_process* pr = procs[g];
    if (!ev || ev->magic != MAGIC_EVT || !pr || pr->magic != MAGIC_PROC || !tfs[g])
      return bfail(MEM_ERR_INVALID_ARG, "group " + std::to_string(g) + ": invalid handle or tf");
    if (ev->kind != pr->desc.kind)
      return bfail(MEM_ERR_INVALID_ARG, "group " + std::to_string(g) + ": process kind mismatch");
    const int kind = pr->desc.kind, d = dims_of(kind), np = nperm_of(kind);
    const mem_tf_desc& T = *tfs[g];
    if ((kind == PROC_DY || kind == PROC_W) &&
        !(T.lep_rel > 0 && T.window_k > 0 && T.lep_rel * T.window_k < 1))
      return bfail(MEM_ERR_INVALID_ARG, "lepton TF parameters invalid");
    if ((kind == PROC_W || kind == PROC_TTBAR) && !(T.met_sigma > 0 && T.met_box_k > 0))
      return bfail(MEM_ERR_INVALID_ARG, "MET TF parameters invalid");
    if ((kind == PROC_TTBAR || kind == PROC_TTDL || kind == PROC_TTH || kind == PROC_TTBB) &&
        !(T.jet_core > 0 && T.jet_tail > 0 && T.jet_tail_w >= 0 && T.jet_tail_w <= 1 &&
          T.jet_lo_div > 1 && T.jet_hi_mul > 1))
      return bfail(MEM_ERR_INVALID_ARG, "jet TF parameters invalid");
    // per-device set-up that may synchronise: before the graph capture below
    if (kind == PROC_TTH || kind == PROC_TTBB) {
      const cudaError_t pe = kind == PROC_TTH ? prepare_tth() : prepare_ttbb();
      if (pe != cudaSuccess)
        return bfail(MEM_ERR_CUDA, std::string("kernel set-up: ") + cudaGetErrorString(pe));
    }
    // this group's schedule: its plan entry where given, else the common options
    const mem_plan* pl = opts->plans ? &opts->plans[g] : nullptr;
    const int iters = pl && pl->n_adapt_iters ? pl->n_adapt_iters : opts->n_adapt_iters;
    if (iters < 1 || iters > 64)
      return bfail(MEM_ERR_INVALID_ARG, "group " + std::to_string(g) + ": n_adapt_iters must be in [1, 64]");
    const uint64_t adapt_pts = pl && pl->adapt_points ? pl->adapt_points
                                                      : (opts->adapt_points ? opts->adapt_points : 8192);
    const uint64_t min_ev = pl && pl->min_points ? pl->min_points
                                                 : (opts->min_points ? opts->min_points : (uint64_t)1 << 14);
    const int tiles = pl && pl->tiles_per_cta ? pl->tiles_per_cta : 4;
    if (adapt_pts > (1u << 24) || tiles < 1 || tiles > 64)
      return bfail(MEM_ERR_INVALID_ARG, "group " + std::to_string(g) + ": plan out of range");
    Plan& p = plans[g];
    BatchArgs& b = p.b;
    IntegrateArgs& a = b.base;
    b.tiles_per_cta = tiles;
    a.recs = ev->d_recs;
    a.n_events = ev->n;
    a.n_items = ev->n * np;
    a.P = pr->pc;
    a.T = make_tf_const_from(&T);
    a.seed = seed;
    a.event_id_base = opts->event_id_base + (uint64_t)ev_total;
    a.n_iters = iters;
    a.n_adapt = (uint32_t)adapt_pts;
    a.alpha = alpha;
    a.grid_in = nullptr;
    a.phase_events = nullptr;
    const uint64_t cap_item = cap_ev / np;
    const uint64_t adapt = (uint64_t)iters * a.n_adapt;
    uint64_t pts0 = (min_ev / np + 255) / 256 * 256;
    pts0 = pts0 < 256 ? 256 : pts0;
    if (cap_item < adapt + pts0)
      return bfail(MEM_ERR_INVALID_ARG, "max_points too small for the adaptation plan and the first round");
    int rounds = 1;
    while (adapt + pts0 * ((((uint64_t)1) << (rounds + 1)) - 1) <= cap_item && rounds < 24) ++rounds;
    if (adapt + pts0 * ((((uint64_t)1) << rounds) - 1) > ((uint64_t)1 << 32))
      return bfail(MEM_ERR_INVALID_ARG, "point budget above 2^32 per item");
    b.kind = kind;
    b.nperm = np;
    b.target = opts->target_rel_err;
    b.n_rounds = rounds;
    b.pts0 = (uint32_t)pts0;
    p.ev_off = ev_total;
    const size_t slots_n = (size_t)a.n_items + 4 * (size_t)sms * 16 + 1024;
    p.off_grid = total; total += up((size_t)a.n_items * d * NG * sizeof(GridBin));
    p.off_cache = total; total += up((size_t)a.n_items * cache_size(kind));
    p.off_acc = total; total += up((size_t)a.n_items * sizeof(ItemAcc));
    p.off_act = total; total += up((size_t)a.n_items * sizeof(int32_t));
    p.off_flags = total; total += up((size_t)a.n_items);
    p.off_ctl = total; total += up(sizeof(RoundCtl));
    p.off_slots = total; total += up(slots_n * sizeof(Slot));
    p.off_state = total; total += up((size_t)a.n_events * sizeof(int32_t));
    ev_total += ev->n;
  }
  const bool dev_out = dev_ptr(prob);
  size_t off_out = total;
  if (!dev_out) total += 4 * up((size_t)ev_total * 8);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&ws, total, st);
  if (e != cudaSuccess) return bfail(e == cudaErrorMemoryAllocation ? MEM_ERR_OOM : MEM_ERR_CUDA, "workspace allocation");
  double* o_prob = dev_out ? prob : reinterpret_cast<double*>(ws + off_out);
  double* o_err = dev_out ? err : reinterpret_cast<double*>(ws + off_out + up((size_t)ev_total * 8));
  uint64_t* o_used = dev_out ? n_used : reinterpret_cast<uint64_t*>(ws + off_out + 2 * up((size_t)ev_total * 8));
  int32_t* o_st = dev_out ? ev_status : reinterpret_cast<int32_t*>(ws + off_out + 3 * up((size_t)ev_total * 8));
  for (auto& p : plans) {
    BatchArgs& b = p.b;
    b.base.grid32 = reinterpret_cast<GridBin*>(ws + p.off_grid);
    b.base.caches = ws + p.off_cache;
    b.acc = reinterpret_cast<ItemAcc*>(ws + p.off_acc);
    b.active = reinterpret_cast<int32_t*>(ws + p.off_act);
    b.flags = ws + p.off_flags;
    b.ctl = reinterpret_cast<RoundCtl*>(ws + p.off_ctl);
    b.slots = reinterpret_cast<Slot*>(ws + p.off_slots);
    b.ev_state = reinterpret_cast<int32_t*>(ws + p.off_state);
    b.prob = o_prob + p.ev_off;
    b.err = o_err + p.ev_off;
    b.n_used = o_used ? o_used + p.ev_off : nullptr;
    b.status = o_st ? o_st + p.ev_off : nullptr;
  }

  // one CUDA graph: every group on its own forked stream, all rounds inside
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> gs(n_groups, nullptr);
  cudaEvent_t fork = nullptr, join = nullptr;
  std::vector<cudaEvent_t> done(n_groups, nullptr);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (int g = 0; g < n_groups && e == cudaSuccess; ++g) {
    e = cudaStreamCreateWithFlags(&gs[g], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[g], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  // the graph starts after prior work on the caller's stream (workspace allocation)
  if (e == cudaSuccess) e = cudaEventRecord(join, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, join, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t ce = cudaEventRecord(fork, cs);
    for (int g = 0; g < n_groups && ce == cudaSuccess; ++g) {
      ce = cudaStreamWaitEvent(gs[g], fork, 0);
      if (ce != cudaSuccess) break;
      const int kind = plans[g].b.kind;
      ce = kind == PROC_DY     ? launch_batch_dy(plans[g].b, gs[g])
           : kind == PROC_W    ? launch_batch_w(plans[g].b, gs[g])
           : kind == PROC_TTDL ? launch_batch_ttdl(plans[g].b, gs[g])
           : kind == PROC_TTH  ? launch_batch_tth(plans[g].b, gs[g])
           : kind == PROC_TTBB ? launch_batch_ttbb(plans[g].b, gs[g])
                               : launch_batch_tt(plans[g].b, gs[g]);
      if (ce == cudaSuccess) ce = cudaEventRecord(done[g], gs[g]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, done[g], 0);
    }
    e = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ce;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
  if (e == cudaSuccess) e = cudaEventRecord(join, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join, 0);
  if (e == cudaSuccess && !dev_out) {
    e = cudaMemcpyAsync(prob, o_prob, ev_total * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err, o_err, ev_total * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n_used) e = cudaMemcpyAsync(n_used, o_used, ev_total * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ev_status) e = cudaMemcpyAsync(ev_status, o_st, ev_total * 4, cudaMemcpyDeviceToHost, st);
  }
  cudaError_t e2 = cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (int g = 0; g < n_groups; ++g) {
    if (gs[g]) cudaStreamDestroy(gs[g]);
    if (done[g]) cudaEventDestroy(done[g]);
  }
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    const std::string m = std::string("mem_integrate_batch: ") + cudaGetErrorString(e);
    mem::set_last_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? MEM_ERR_OOM : MEM_ERR_CUDA;
  }
  return MEM_OK;
}
