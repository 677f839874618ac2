// Adaptive-budget integration (per-event stop rule at a target relative error)
// for batches of uneven events, as fixed rounds of device-side work.
//
// After the adaptation kernel (grids + per-item constants), round r gives every
// still-active item P_r = P_0 2^r more frozen-grid points:
//   k_round_sample : persistent CTAs walk the compacted list of active items in
//                    tiles; the tile count per item is chosen on the device from
//                    the active count (>= ~4 tiles per CTA), each tile writes one
//                    slot at a fixed position (deterministic).
//   k_round_reduce : per active item, its slots in order -> running FP64 sums.
//   k_round_check  : per event, the estimate over permutations (Sec. 4: average)
//                    and its MC error (Sec. 2); done when err <= target |p| or the
//                    next round would pass the point cap. Within an unconverged
//                    event only the items whose variance still matters go on
//                    (a cheap form of allocating points in proportion to sigma).
//   k_round_compact: one CTA, prefix scan of the active flags -> next active list.
// Every round's launch sequence is fixed, so all rounds of all processes are
// captured into one CUDA graph; no host synchronisation between rounds.
#pragma once
#include "mem_internal.h"
#include "mem_kernels.cuh"

namespace mem {

struct ItemAcc {
  double s1, c1, s2, c2;  // running sum w, sum w^2 (double-word)
  uint64_t n;             // frozen-grid points accumulated
  uint32_t n_bad, pad;
};

struct RoundCtl {
  int32_t n_active;       // active items this round
  int32_t tiles_per_item;
  int32_t n_events_active;
  int32_t pad;
};

__device__ __forceinline__ void neu2(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

template <class PH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_round_sample(const float* __restrict__ recs, ProcConst P, const __grid_constant__ PhiloxKey key,
               uint64_t event_id_base, const int32_t* __restrict__ active,
               const RoundCtl* __restrict__ ctl, uint32_t idx_base, uint32_t pts_item,
               const GridBin* __restrict__ grid32, const typename PH::Cache* __restrict__ caches,
               Slot* __restrict__ slots) {
  constexpr int D = PH::D;
  __shared__ MainSmem<PH> S;
  const int n_act = ctl->n_active, tpi = ctl->tiles_per_item;
  const int64_t n_tiles = (int64_t)n_act * tpi;
  const uint32_t per_tile = ((pts_item + tpi - 1) / tpi + THREADS - 1) / THREADS * THREADS;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int32_t item = active[tile / tpi];
    const uint32_t k = (uint32_t)(tile % tpi);
    const int64_t ev = item / PH::NPERM;
    const int perm = (int)(item % PH::NPERM);
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(caches + item);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&S.cache);
      for (int t = threadIdx.x; t < (int)(sizeof(typename PH::Cache) / 4); t += blockDim.x)
        dst[t] = src[t];
      const GridBin* gsrc = grid32 + (int64_t)item * (D * NG);
      for (int t = threadIdx.x; t < D * NG; t += blockDim.x) S.gb[t] = gsrc[t];
    }
    __syncthreads();
    const uint32_t eid = (uint32_t)(event_id_base + (uint64_t)ev);
    const uint32_t p0 = k * per_tile;
    const uint32_t p1 = min(p0 + per_tile, pts_item);
    Kahan32 a1, a2;
    uint32_t nbad = 0;
    if (S.cache.ok) {
#pragma unroll 1
      for (uint32_t p = p0 + threadIdx.x; p < p1; p += THREADS) {
        float u[D], x[D], xc[D];
        int bin[D];
        point_uniforms<D>(key, eid, (uint32_t)perm, idx_base + p, u);
        const float J = vegas_map<D>(S.gb, u, x, xc, bin);
        const float w = PH::eval(S.cache, P, x, xc) * J;
        if (isfinite(w)) {
          a1.add(w);
          a2.add(w * w);
        } else {
          ++nbad;
        }
      }
    }
    const DD v1 = warp_reduce_kahan(a1), v2 = warp_reduce_kahan(a2);
    for (int o = 16; o > 0; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      S.red[0][warp] = v1;
      S.red[1][warp] = v2;
      S.bad[warp] = nbad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      DD s1 = S.red[0][0], s2 = S.red[1][0];
      uint32_t b = S.bad[0];
      for (int w = 1; w < WARPS; ++w) {
        s1 = two_sum_merge(s1, S.red[0][w]);
        s2 = two_sum_merge(s2, S.red[1][w]);
        b += S.bad[w];
      }
      Slot sl;
      sl.s1 = s1.hi;
      sl.c1 = s1.lo;
      sl.s2 = s2.hi;
      sl.c2 = s2.lo;
      sl.n_bad = b | (S.cache.ok ? 0u : 0x80000000u);
      sl.pad = 0;
      slots[tile] = sl;
    }
    __syncthreads();
  }
}

// Per active item: add its tiles' slots (in order) to the running sums.
__global__ void k_round_reduce(const int32_t* __restrict__ active, const RoundCtl* __restrict__ ctl,
                               uint32_t pts_item, const Slot* __restrict__ slots,
                               ItemAcc* __restrict__ acc);

// Per event: estimate, error, stop rule; writes item active flags (only the
// items of an unconverged event whose variance still matters stay active).
__global__ void k_round_check(int64_t n_events, int nperm, double target, double prefactor,
                              int last_round, uint64_t keep_n, const ItemAcc* __restrict__ acc,
                              int32_t* __restrict__ ev_state, uint8_t* __restrict__ flags);

// One CTA: active flags -> compacted list, counts and tiles per item. With
// sel != nullptr only items with sel[i] == want are listed.
__global__ void k_round_compact(int64_t n_items, const uint8_t* __restrict__ flags,
                                int32_t* __restrict__ active, RoundCtl* __restrict__ ctl,
                                int target_tiles, const uint8_t* __restrict__ sel, int want);

// Final per-event outputs from the running sums. Every item's adaptation
// points count as used, or with adapted != nullptr only those of items with
// adapted[i] != 0.
__global__ void k_batch_final(int64_t n_events, int nperm, double prefactor, uint64_t adapt_pts_item,
                              const ItemAcc* __restrict__ acc, const int32_t* __restrict__ ev_state,
                              const uint8_t* __restrict__ adapted, double* __restrict__ prob,
                              double* __restrict__ err, uint64_t* __restrict__ n_used,
                              int32_t* __restrict__ status);

// Buffers and schedule of one process group.
struct BatchArgs {
  IntegrateArgs base;        // recs, P, T, seed, ids, adaptation plan, grid32, caches
  int kind, nperm;
  double target;
  int n_rounds;
  uint32_t pts0;             // frozen-grid points per item in round 0
  ItemAcc* acc;
  int32_t* active;
  uint8_t* flags;
  RoundCtl* ctl;
  Slot* slots;
  int32_t* ev_state;         // 0 active, 1 converged, 2 cap reached, 3 invalid record
  int grid_ctas;             // persistent sampling CTAs
  int tiles_per_cta;         // sampling tiles per CTA and round
  int target_tiles;
  double* prob;              // device outputs of this group (n_events each)
  double* err;
  uint64_t* n_used;
  int32_t* status;
};


template <class PH, int MINB>
int round_sample_ctas() {
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_round_sample<PH, MINB>, THREADS, 0);
  return (per_sm > 0 ? per_sm : 1) * sms;
}

template <class PH, int MINB>
cudaError_t run_batch_rounds(const BatchArgs& b, cudaStream_t st) {
  uint32_t idx = (uint32_t)((uint64_t)b.base.n_iters * b.base.n_adapt);
  uint32_t pts = b.pts0;
  for (int r = 0; r < b.n_rounds; ++r) {
    k_round_sample<PH, MINB><<<b.grid_ctas, THREADS, 0, st>>>(
        b.base.recs, b.base.P, philox_key(b.base.seed), b.base.event_id_base, b.active, b.ctl, idx, pts,
        b.base.grid32, reinterpret_cast<const typename PH::Cache*>(b.base.caches), b.slots);
    k_round_reduce<<<(unsigned)((b.base.n_items + 255) / 256), 256, 0, st>>>(b.active, b.ctl, pts,
                                                                            b.slots, b.acc);
    k_round_check<<<(unsigned)((b.base.n_events + 127) / 128), 128, 0, st>>>(
        b.base.n_events, b.nperm, b.target, b.base.P.prefactor, r == b.n_rounds - 1,
        (uint64_t)b.pts0 * 4, b.acc, b.ev_state, b.flags);
    k_round_compact<<<1, 1024, 0, st>>>(b.base.n_items, b.flags, b.active, b.ctl, b.target_tiles,
                                        nullptr, 0);
    idx += pts;
    pts *= 2;
  }
  return cudaGetLastError();
}

// Enqueue one group's whole schedule on `st`: adaptation, rounds, outputs.
template <class PH, int MINB>
cudaError_t run_batch(BatchArgs b, cudaStream_t st) {
  const size_t smem = sizeof(AdaptSmem<PH>);
  cudaError_t e = cudaFuncSetAttribute(k_adapt<PH, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const IntegrateArgs& a = b.base;
  k_adapt<PH, MINB><<<(unsigned)a.n_items, THREADS, smem, st>>>(
      a.recs, a.P, a.T, a.n_items, philox_key(a.seed), a.event_id_base, a.n_iters, a.n_adapt, a.alpha,
      a.grid_in, a.grid32, reinterpret_cast<typename PH::Cache*>(a.caches));
  b.grid_ctas = round_sample_ctas<PH, MINB>();
  b.target_tiles = b.tiles_per_cta * b.grid_ctas;
  cudaMemsetAsync(b.flags, 1, (size_t)a.n_items, st);
  cudaMemsetAsync(b.acc, 0, (size_t)a.n_items * sizeof(ItemAcc), st);
  cudaMemsetAsync(b.ev_state, 0, (size_t)a.n_events * sizeof(int32_t), st);
  k_round_compact<<<1, 1024, 0, st>>>(a.n_items, b.flags, b.active, b.ctl, b.target_tiles, nullptr,
                                      0);
  e = run_batch_rounds<PH, MINB>(b, st);
  if (e != cudaSuccess) return e;
  k_batch_final<<<(unsigned)((a.n_events + 127) / 128), 128, 0, st>>>(
      a.n_events, b.nperm, a.P.prefactor, (uint64_t)a.n_iters * a.n_adapt, b.acc, b.ev_state,
      nullptr, b.prob, b.err, b.n_used, b.status);
  return cudaGetLastError();
}

}  // namespace mem
