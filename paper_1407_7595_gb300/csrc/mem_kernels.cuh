// Integration kernels, templated on the process physics (PhysDY, PhysW, PhysTT).
//
// One item = (event, jet permutation). Per item:
//   k_adapt : one CTA runs the VEGAS adaptation iterations (Sec. 2, Lepage's
//             algorithm): Philox points -> grid map -> integrand -> squared
//             weights histogrammed in shared memory -> FP64 grid refinement
//             (one warp per dimension) -> next iteration. Leaves the frozen
//             FP32 grid of the item in global memory.
//   k_main  : CTAs of CHUNK points each sample the frozen grid; each thread
//             keeps FP32 Kahan sums of w and w^2, merged by FP64 TwoSum warp
//             shuffles and a fixed-order CTA reduction into one slot.
//   k_final : one thread per event reduces its slots in fixed order (FP64
//             Neumaier), forms the plain MC mean and error (Sec. 2, Eq. "sum"),
//             averages over permutations (Sec. 4) and applies the FP64 prefactor.
#pragma once
#include "mem_physics.cuh"

namespace mem {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;

// ---------------------------------------------------------------------------
// VEGAS refinement of one dimension by one warp (Lepage 1978): three-point
// smoothing of the bin importances h, normalisation, compression
// w_i = ((1 - r_i)/ln(1/r_i))^alpha, re-binning to equal w per bin.
// g: NG+1 edges (updated in place); h: NG importances; wk, cum: scratch.
// Precision: importances, their sums and the new edges in FP64; the
// compression exponent (a damping heuristic whose rounding moves edges by
// ~1e-7 of a bin and cannot bias the estimate) in FP32, because FP64
// transcendentals run at a small fraction of the FP32 rate on this part.
// Each lane owns NG/32 consecutive bins; sums are warp scans.
// ---------------------------------------------------------------------------
__device__ inline void refine_dim_warp(double* g, const double* h, double* wk, double* cum,
                                       double* newg, double alpha) {
  static_assert(NG % 32 == 0, "bins per lane");
  constexpr int BPL = NG / 32;
  const int lane = threadIdx.x & 31;
  const int i0 = lane * BPL;
  double sm[BPL];
  double part = 0.0;
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    const int i = i0 + q;
    double s;
    if (i == 0) s = 0.5 * (h[0] + h[1]);
    else if (i == NG - 1) s = 0.5 * (h[NG - 2] + h[NG - 1]);
    else s = (h[i - 1] + h[i] + h[i + 1]) * (1.0 / 3.0);
    sm[q] = s;
    part += s;
  }
  double tot = part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if (!(tot > 0.0)) return;
  const double inv = 1.0 / tot;
  const float af = (float)alpha;
  double wsum = 0.0;
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    const double r = sm[q] * inv;
    double w;
    if (!(r > 0.0)) {
      w = 0.0;
    } else if (r >= 1.0) {
      w = 1.0;
    } else {
      const float rf = fmaxf((float)r, 1e-30f);
      w = (double)powf((1.f - rf) / -logf(rf), af);
    }
    sm[q] = w;
    wsum += w;
  }
  // exclusive prefix of the lane sums
  double incl = wsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  double acc = incl - wsum;
#pragma unroll
  for (int q = 0; q < BPL; ++q) {
    wk[i0 + q] = sm[q];
    cum[i0 + q] = acc;
    acc += sm[q];
  }
  if (lane == 31) cum[NG] = incl;
  __syncwarp();
  const double per = cum[NG] * (1.0 / NG);
  for (int k = lane; k <= NG; k += 32) {
    double e;
    if (k == 0 || k == NG) {
      e = g[k];
    } else {
      const double target = k * per;
      // smallest i with cum[i] + w[i] >= target (i <= NG - 1)
      int lo = 0, hi = NG - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cum[mid] + wk[mid] < target) lo = mid + 1;
        else hi = mid;
      }
      const int i = lo;
      double frac = wk[i] > 0.0 ? (target - cum[i]) / wk[i] : 0.0;
      frac = frac < 0.0 ? 0.0 : (frac > 1.0 ? 1.0 : frac);
      e = g[i] + frac * (g[i + 1] - g[i]);
    }
    newg[k] = e;
  }
  __syncwarp();
  for (int k = lane; k <= NG; k += 32) g[k] = newg[k];
  __syncwarp();
}

template <int D>
__device__ inline void grid_to_bins(const double* g /* D x (NG+1) */, GridBin* gb) {
  for (int t = threadIdx.x; t < D * NG; t += blockDim.x) {
    const int j = t / NG, i = t % NG;
    const double a = g[j * (NG + 1) + i], b = g[j * (NG + 1) + i + 1];
    gb[t].x0 = (float)a;
    gb[t].w = (float)(b - a);
    gb[t].xc = (float)(1.0 - b);
    gb[t].pad = 0.f;
  }
}

template <class PH>
struct AdaptSmem {
  typename PH::Cache cache;
  double g[PH::D * (NG + 1)];
  double h[PH::D * NG];
  double wk[PH::D * NG];
  double cum[PH::D * (NG + 1)];
  double newg[PH::D * (NG + 1)];
  GridBin gb[PH::D * NG];
  float hist[PH::D * NG];
  DD red[2][WARPS];
};

// One CTA adapts the VEGAS grid of one item: n_iters iterations of n_adapt
// points, each filling the per-bin histograms of w^2 and refining every
// dimension (one warp per dimension, FP64). With MOM, the moments of the last
// iteration (sum w, sum w^2, compensated) are written to *mom: the variance of
// the sampler the adapted grid replaces, for comparing samplers (the per-item
// constants are then read from `caches`, filled by the caller). With hist0,
// the starting grid is first refined once with the item's histogram
// hist0[item] (D x NG sums of w^2 over bins of the starting grid, gathered by
// another sampler).
template <class PH, bool MOM>
__device__ void adapt_item(AdaptSmem<PH>& S, const float* __restrict__ recs, const ProcConst& P,
                           const TFConst& T, int64_t item, const PhiloxKey& key, uint64_t event_id_base,
                           int n_iters, uint32_t n_adapt, double alpha,
                           const double* __restrict__ grid_in, GridBin* __restrict__ grid32,
                           typename PH::Cache* __restrict__ caches, Slot* __restrict__ mom,
                           const float* __restrict__ hist0 = nullptr) {
  constexpr int D = PH::D;
  const int64_t ev = item / PH::NPERM;
  const int perm = (int)(item % PH::NPERM);
  const float* rec = recs + ev * REC;
  if (MOM) {
    // the judge of another sampler: the per-item constants are already in HBM
    static_assert(sizeof(typename PH::Cache) % 4 == 0, "cache must be word sized");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(caches + item);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&S.cache);
    for (int t = threadIdx.x; t < (int)(sizeof(typename PH::Cache) / 4); t += blockDim.x)
      dst[t] = src[t];
  } else if (threadIdx.x == 0) {
    // per-item constants, computed once in FP64 and kept for the sampling kernel
    PH::setup(rec, perm, P, T, S.cache);
    caches[item] = S.cache;
  }
  for (int t = threadIdx.x; t < D * (NG + 1); t += blockDim.x)
    S.g[t] = grid_in ? grid_in[t] : (double)(t % (NG + 1)) / NG;
  __syncthreads();
  if (hist0) {
    for (int t = threadIdx.x; t < D * NG; t += blockDim.x) S.h[t] = (double)hist0[item * (D * NG) + t];
    __syncthreads();
    for (int j = threadIdx.x >> 5; j < D; j += WARPS)
      refine_dim_warp(S.g + j * (NG + 1), S.h + j * NG, S.wk + j * NG, S.cum + j * (NG + 1),
                      S.newg + j * (NG + 1), alpha);
    __syncthreads();
  }
  grid_to_bins<D>(S.g, S.gb);
  const uint32_t eid = (uint32_t)(event_id_base + (uint64_t)ev);
  Kahan32 a1, a2;
  for (int it = 0; it < n_iters; ++it) {
    for (int t = threadIdx.x; t < D * NG; t += blockDim.x) S.hist[t] = 0.f;
    __syncthreads();
    if (S.cache.ok) {
      for (uint32_t k = threadIdx.x; k < n_adapt; k += blockDim.x) {
        float u[D], x[D], xc[D];
        int bin[D];
        point_uniforms<D>(key, eid, (uint32_t)perm, (uint32_t)it * n_adapt + k, u);
        const float J = vegas_map<D>(S.gb, u, x, xc, bin);
        const float w = PH::eval(S.cache, P, x, xc) * J;
        if (isfinite(w)) {
          const float w2 = w * w;
#pragma unroll
          for (int j = 0; j < D; ++j) atomicAdd(&S.hist[j * NG + bin[j]], w2);
          if (MOM && it == n_iters - 1) {
            a1.add(w);
            a2.add(w2);
          }
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < D * NG; t += blockDim.x) S.h[t] = (double)S.hist[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    for (int j = warp; j < D; j += WARPS)
      refine_dim_warp(S.g + j * (NG + 1), S.h + j * NG, S.wk + j * NG, S.cum + j * (NG + 1),
                      S.newg + j * (NG + 1), alpha);
    __syncthreads();
    grid_to_bins<D>(S.g, S.gb);
    __syncthreads();
  }
  GridBin* out = grid32 + item * (D * NG);
  for (int t = threadIdx.x; t < D * NG; t += blockDim.x) out[t] = S.gb[t];
  if (MOM) {
    const DD v1 = warp_reduce_kahan(a1), v2 = warp_reduce_kahan(a2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      S.red[0][warp] = v1;
      S.red[1][warp] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      DD s1 = S.red[0][0], s2 = S.red[1][0];
      for (int w = 1; w < WARPS; ++w) {
        s1 = two_sum_merge(s1, S.red[0][w]);
        s2 = two_sum_merge(s2, S.red[1][w]);
      }
      Slot sl;
      sl.s1 = s1.hi;
      sl.c1 = s1.lo;
      sl.s2 = s2.hi;
      sl.c2 = s2.lo;
      sl.n_bad = S.cache.ok ? 0u : 0x80000000u;
      sl.pad = 0;
      *mom = sl;
    }
  }
  __syncthreads();
}

template <class PH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_adapt(const float* __restrict__ recs, ProcConst P, TFConst T, int64_t n_items,
        const __grid_constant__ PhiloxKey key, uint64_t event_id_base, int n_iters, uint32_t n_adapt, double alpha,
        const double* __restrict__ grid_in, GridBin* __restrict__ grid32,
        typename PH::Cache* __restrict__ caches) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AdaptSmem<PH>& S = *reinterpret_cast<AdaptSmem<PH>*>(smem_raw);
  const int64_t item = blockIdx.x;
  if (item >= n_items) return;
  adapt_item<PH, false>(S, recs, P, T, item, key, event_id_base, n_iters, n_adapt, alpha,
                        grid_in, grid32, caches, nullptr);
}

// Adaptation of the items in list[0 .. *n_list) (persistent CTAs), with the
// last iteration's moments per item in mom[item] and an optional starting
// histogram per item (hist0, see adapt_item).
template <class PH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_adapt_list(const float* __restrict__ recs, ProcConst P, TFConst T,
             const int32_t* __restrict__ list, const int32_t* __restrict__ n_list,
             const __grid_constant__ PhiloxKey key,
             uint64_t event_id_base, int n_iters, uint32_t n_adapt, double alpha,
             GridBin* __restrict__ grid32, typename PH::Cache* __restrict__ caches,
             Slot* __restrict__ mom, const float* __restrict__ hist0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AdaptSmem<PH>& S = *reinterpret_cast<AdaptSmem<PH>*>(smem_raw);
  const int n = *n_list;
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int64_t item = list[b];
    adapt_item<PH, true>(S, recs, P, T, item, key, event_id_base, n_iters, n_adapt, alpha,
                         nullptr, grid32, caches, mom + item, hist0);
  }
}

template <class PH>
struct MainSmem {
  typename PH::Cache cache;
  GridBin gb[PH::D * NG];
  DD red[2][WARPS];
  uint32_t bad[WARPS];
};

// Sample the frozen grid: CTA b handles points [chunk*CHUNK, (chunk+1)*CHUNK)
// of item b / chunks_per_item, main-phase point index offset idx0.
template <class PH, int PPT, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_main(const float* __restrict__ recs, ProcConst P, TFConst T, int64_t n_items,
       uint32_t chunks_per_item, const __grid_constant__ PhiloxKey key, uint64_t event_id_base,
       uint32_t idx0,
       uint32_t n_main, const GridBin* __restrict__ grid32,
       const typename PH::Cache* __restrict__ caches, Slot* __restrict__ slots) {
  constexpr int D = PH::D;
  constexpr uint32_t CHUNK = THREADS * PPT;
  __shared__ MainSmem<PH> S;
  const int64_t item = blockIdx.x / chunks_per_item;
  const uint32_t chunk = blockIdx.x % chunks_per_item;
  if (item >= n_items) return;
  const int64_t ev = item / PH::NPERM;
  const int perm = (int)(item % PH::NPERM);
  {
    static_assert(sizeof(typename PH::Cache) % 4 == 0, "cache must be word sized");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(caches + item);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&S.cache);
    for (int t = threadIdx.x; t < (int)(sizeof(typename PH::Cache) / 4); t += blockDim.x)
      dst[t] = src[t];
  }
  const GridBin* gsrc = grid32 + item * (D * NG);
  for (int t = threadIdx.x; t < D * NG; t += blockDim.x) S.gb[t] = gsrc[t];
  __syncthreads();
  const uint32_t eid = (uint32_t)(event_id_base + (uint64_t)ev);
  Kahan32 a1, a2;
  uint32_t nbad = 0;
  if (S.cache.ok) {
    const uint32_t base = chunk * CHUNK;
#pragma unroll 1
    for (int j = 0; j < PPT; ++j) {
      const uint32_t p = base + (uint32_t)j * THREADS + threadIdx.x;
      if (p < n_main) {
        float u[D], x[D], xc[D];
        int bin[D];
        point_uniforms<D>(key, eid, (uint32_t)perm, idx0 + p, u);
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
  }
  // Kahan state (s, c) represents s - c
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
    slots[blockIdx.x] = sl;
  }
}

// Stratified frozen-grid sampling (Sec. 4: the VEGAS integrator's stratified
// sampling): the map's input cube is divided into M = ns^D equal hypercubes with
// k points each; hypercube c has the base-ns digits of c as coordinates
// (dimension 0 least significant) and its points the Philox indices
// idx0 + c k + i. Thread t of CTA (item, chunk) takes hypercubes
// chunk CPC + j THREADS + t, j < cubes_per_thread (CPC = THREADS cubes_per_thread),
// and accumulates the per-cube mean into a1 and the per-cube sample variance / k
// into a2 (Welford within the hypercube); non-finite weights count as 0 and are
// reported.
template <class PH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_main_strat(const float* __restrict__ recs, ProcConst P, TFConst T, int64_t n_items,
             uint32_t chunks_per_item, const __grid_constant__ PhiloxKey key,
             uint64_t event_id_base, uint32_t idx0, uint32_t ns, uint32_t n_cubes, uint32_t k,
             uint32_t cubes_per_thread, const GridBin* __restrict__ grid32,
             const typename PH::Cache* __restrict__ caches, Slot* __restrict__ slots) {
  constexpr int D = PH::D;
  __shared__ MainSmem<PH> S;
  const int64_t item = blockIdx.x / chunks_per_item;
  const uint32_t chunk = blockIdx.x % chunks_per_item;
  if (item >= n_items) return;
  const int64_t ev = item / PH::NPERM;
  const int perm = (int)(item % PH::NPERM);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(caches + item);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&S.cache);
    for (int t = threadIdx.x; t < (int)(sizeof(typename PH::Cache) / 4); t += blockDim.x)
      dst[t] = src[t];
  }
  const GridBin* gsrc = grid32 + item * (D * NG);
  for (int t = threadIdx.x; t < D * NG; t += blockDim.x) S.gb[t] = gsrc[t];
  __syncthreads();
  const uint32_t eid = (uint32_t)(event_id_base + (uint64_t)ev);
  Kahan32 a1, a2;
  uint32_t nbad = 0;
  if (S.cache.ok) {
    const float inv_ns = 1.f / (float)ns;
    const float below_one = 0x1.fffffep-1f;
    const uint32_t cube0 = chunk * (THREADS * cubes_per_thread);
    const float inv_kk = 1.f / ((float)(k - 1) * (float)k);
#pragma unroll 1
    for (uint32_t j = 0; j < cubes_per_thread; ++j) {
      const uint32_t c = cube0 + j * THREADS + threadIdx.x;
      if (c >= n_cubes) break;
      float cell[D];
      uint32_t r = c;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const uint32_t t = r / ns;
        cell[q] = (float)(r - t * ns);
        r = t;
      }
      float mean = 0.f, m2 = 0.f;
#pragma unroll 1
      for (uint32_t i = 0; i < k; ++i) {
        float u[D], x[D], xc[D];
        int bin[D];
        point_uniforms<D>(key, eid, (uint32_t)perm, idx0 + c * k + i, u);
#pragma unroll
        for (int q = 0; q < D; ++q) u[q] = fminf((cell[q] + u[q]) * inv_ns, below_one);
        const float J = vegas_map<D>(S.gb, u, x, xc, bin);
        float w = PH::eval(S.cache, P, x, xc) * J;
        if (!isfinite(w)) {
          ++nbad;
          w = 0.f;
        }
        const float delta = w - mean;
        mean += delta / (float)(i + 1);
        m2 = fmaf(delta, w - mean, m2);
      }
      a1.add(mean);
      a2.add(m2 * inv_kk);
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
    slots[blockIdx.x] = sl;
  }
}

// Per event: fixed-order FP64 reduction of the item slots, MC mean and error
// per item, average over permutations, FP64 prefactor.
__global__ void k_final(const Slot* __restrict__ slots, int64_t n_events, int nperm,
                        uint32_t chunks_per_item, uint32_t n_main, uint64_t n_per_item,
                        uint32_t n_cubes, double prefactor, double* __restrict__ prob,
                        double* __restrict__ err, uint64_t* __restrict__ n_used,
                        int32_t* __restrict__ status);

// Integrand at consecutive points of one item (parity tests): one thread per point.
template <class PH>
__global__ void __launch_bounds__(THREADS)
k_eval(const float* __restrict__ rec, int perm, ProcConst P, TFConst T,
       const __grid_constant__ PhiloxKey key,
       uint32_t event_id, uint32_t point0, int64_t n, const GridBin* __restrict__ gb,
       double* __restrict__ w_out) {
  constexpr int D = PH::D;
  __shared__ typename PH::Cache cache;
  __shared__ GridBin sg[D * NG];
  if (threadIdx.x == 0) PH::setup(rec, perm, P, T, cache);
  for (int t = threadIdx.x; t < D * NG; t += blockDim.x) sg[t] = gb[t];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float u[D], x[D], xc[D];
  int bin[D];
  point_uniforms<D>(key, event_id, (uint32_t)perm, point0 + (uint32_t)i, u);
  const float J = vegas_map<D>(sg, u, x, xc, bin);
  const float w = cache.ok ? PH::eval(cache, P, x, xc) * J : 0.f;
  w_out[i] = (double)w * P.prefactor;
}

}  // namespace mem
