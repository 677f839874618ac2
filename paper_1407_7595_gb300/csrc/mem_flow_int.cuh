// The learned sampler inside the Monte Carlo integral (Sec. 2, importance
// sampling) of the ttbar process: per-item conditioning features, the training
// set drawn from adapted VEGAS grids, and the fused sampling kernel
//
//   Philox u (stream 2) -> z = logit u -> 6 coupling layers (BF16 mma) ->
//   y = sigmoid z -> w = F(y) |dy/du|
//
// whose per-point weight is unbiased for the integral whatever the flow's
// parameters, because |dy/du| is the exact Jacobian of the map that was applied.
//
// The coupling MLPs run on the tensor cores: per 128-point tile and layer, one
// thread issues tcgen05.mma (BF16 operands in shared memory, FP32 accumulators
// in tensor memory, biases folded into the products) for the first (K 16) and
// hidden (K 144) layers; the warps read the accumulators back (tcgen05.ld),
// apply ReLU and repack BF16 operands for the next product. The output layer
// (N 8) runs per warp on mma.sync, where its small N costs less than a
// tensor-memory round trip.
#pragma once
#include "mem_batch.cuh"
#include "mem_flow.cuh"
#include "mem_ttbar.cuh"
#include "mem_umma.cuh"

namespace mem {

constexpr int FCH = 768;         // points per pass of a sampling CTA (z state in shared memory)
constexpr int FROWS = 128;       // rows per tensor-core tile (M of the MMA)
// tensor memory of a CTA: 128 x 128 FP32, the first-layer accumulator and then
// the hidden layer's
constexpr uint32_t F_TMEM_COLS = 128;
constexpr uint32_t F_WAIT_LIMIT = 1u << 20;   // polls of one MMA-completion wait (default)
constexpr uint32_t F_DRAIN_LIMIT = 1u << 22;  // polls of the drain wait after a wait gave up
// Poll limit of the MMA-completion waits of the flow kernels on this device
// (mem_set_tc_wait_limit; tests lower it to exercise the timeout path).
__constant__ uint32_t c_tc_wait_limit = F_WAIT_LIMIT;
constexpr int FTS = 128;         // training samples per item

// The 16 conditioning features of an item (event record, jet permutation), in
// units of 100 GeV, in the frame rotated about the beam so that the lepton has
// phi = 0: lepton (px, pz); jets b, bbar, d, ubar of the permutation, each
// (px, py, pz); missing pT (x, y). Massless objects: pT = E / cosh(eta),
// pz = E tanh(eta).
__device__ inline void flow_features(const float* rec, int perm, float* c) {
  int p[4];
  tt_perm_decode(perm, p);
  const double El = rec[0], etal = rec[1], phil = rec[2];
  const double cl = cos(phil), sl = sin(phil);
  c[0] = (float)(El / cosh(etal) * 0.01);
  c[1] = (float)(El * tanh(etal) * 0.01);
  for (int k = 0; k < 4; ++k) {
    const int o = 1 + p[k];
    const double E = rec[4 * o], eta = rec[4 * o + 1], dphi = (double)rec[4 * o + 2] - phil;
    const double pt = E / cosh(eta);
    c[2 + 3 * k] = (float)(pt * cos(dphi) * 0.01);
    c[3 + 3 * k] = (float)(pt * sin(dphi) * 0.01);
    c[4 + 3 * k] = (float)(E * tanh(eta) * 0.01);
  }
  const double mx = rec[24], my = rec[25];
  c[14] = (float)((mx * cl + my * sl) * 0.01);
  c[15] = (float)((my * cl - mx * sl) * 0.01);
}

// One thread per item: integrand constants and conditioning features.
template <class PH>
__global__ void k_flow_setup(const float* __restrict__ recs, ProcConst P, TFConst T,
                             int64_t n_items, typename PH::Cache* __restrict__ caches,
                             float* __restrict__ feats) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= n_items) return;
  const int64_t ev = item / PH::NPERM;
  const int perm = (int)(item % PH::NPERM);
  const float* rec = recs + ev * REC;
  typename PH::Cache c;
  PH::setup(rec, perm, P, T, c);
  caches[item] = c;
  flow_features(rec, perm, feats + item * FC);
}

// Training set: per item FTS points of the VEGAS stream after the adaptation
// (indices idx0 ..), drawn from the item's adapted grid: y = x, raw weights
// w = F(x) J (samples of F / I, importance-weighted against the VEGAS density),
// their per-item sums in tot[item], and log J (optional); y is kept inside
// [2^-24, 1 - 2^-24] for the logit.
template <class PH>
__global__ void __launch_bounds__(FTS)
k_flow_samples(const float* __restrict__ recs, ProcConst P, int64_t n_items,
               const __grid_constant__ PhiloxKey key,
               uint64_t event_id_base, uint32_t idx0, const GridBin* __restrict__ grid32,
               const typename PH::Cache* __restrict__ caches, float* __restrict__ ys,
               float* __restrict__ ws, float* __restrict__ cs, double* __restrict__ tot_out,
               float* __restrict__ logj) {
  constexpr int D = PH::D;
  __shared__ typename PH::Cache cache;
  __shared__ GridBin gb[D * NG];
  __shared__ double red[FTS / 32];
  const int64_t item = blockIdx.x;
  if (item >= n_items) return;
  const int64_t ev = item / PH::NPERM;
  const int perm = (int)(item % PH::NPERM);
  if (threadIdx.x == 0) cache = caches[item];
  for (int t = threadIdx.x; t < D * NG; t += blockDim.x) gb[t] = grid32[item * (D * NG) + t];
  __syncthreads();
  float u[D], x[D], xc[D];
  int bin[D];
  point_uniforms<D>(key, (uint32_t)(event_id_base + (uint64_t)ev), (uint32_t)perm,
                    idx0 + threadIdx.x, u);
  const float J = vegas_map<D>(gb, u, x, xc, bin);
  float w = cache.ok ? PH::eval(cache, P, x, xc) * J : 0.f;
  if (!isfinite(w) || w < 0.f) w = 0.f;
  double s = w;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  const int64_t row = item * FTS + threadIdx.x;
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < FTS / 32; ++k) tot += red[k];
    tot_out[item] = tot;
  }
  ws[row] = w;
  if (logj) logj[row] = __logf(J);
  const float lo = 5.9604645e-8f, hi = 1.f - 5.9604645e-8f;  // 2^-24, 1 - 2^-24
#pragma unroll
  for (int j = 0; j < D; ++j) ys[row * D + j] = xc[j] < lo ? hi : fmaxf(x[j], lo);
  if (threadIdx.x == 0) flow_features(recs + ev * REC, perm, cs + item * FC);
}

// Weights of the training set normalised to sum 1 per item (per_event = 0) or
// per event (per_event = 1: an item then carries its share of the event's
// estimate, so the loss favours the permutations that dominate the integral).
__global__ void k_flow_normalise(int64_t n_items, int nperm, int per_event,
                                 const double* __restrict__ tot, float* __restrict__ ws) {
  const int64_t item = blockIdx.x;
  if (item >= n_items) return;
  double T = tot[item];
  if (per_event) {
    const int64_t e0 = item / nperm * nperm;
    T = 0.0;
    for (int p = 0; p < nperm; ++p) T += tot[e0 + p];
  }
  const float scale = T > 0.0 ? (float)(1.0 / T) : 0.f;
  for (int t = threadIdx.x; t < FTS; t += blockDim.x) ws[item * FTS + t] *= scale;
}

// Shared memory of a sampling CTA (about 114 KB: two CTAs per SM; tensor
// memory 128 columns each). The tcgen05 operands use the K-major layout of
// umma_kmajor.
template <class PH>
struct __align__(1024) FlowSampSmem {
  __nv_bfloat16 W2u[FH * FKH];    // hidden layer with its bias (B, N 128 x K 144)
  __nv_bfloat16 Act[FROWS * FKH]; // hidden-layer input (+ constant columns), then output-layer input
  __nv_bfloat16 A1[FROWS * 16];   // first-layer input: [z_A hi | z_A lo | z_A hi | 1 1 0 0] per row
  __nv_bfloat16 W1u[FH * 16];     // first layer (B, N 128 x K 16, split form, item bias in K 12-13)
  __nv_bfloat16 W3t[8][FLD];      // output layer, mma.sync B fragments
  float b3[16];
  float zs[FCH * 8];              // per point: z[0..6], running log-Jacobian
  typename PH::Cache cache;
  float c[FC];
  DD red[2][WARPS];
  uint32_t bad[WARPS];
  float hist[PH::D * NG];         // w^2 over NG uniform bins per dimension (pilot round)
  unsigned long long mbar;        // MMA completion
  uint32_t tmem;                  // tensor-memory base address
  int abort;
};

__device__ __forceinline__ void sigmoid_pair(float z, float& y, float& yc, float& lsp) {
  // y = 1/(1+e^-z), 1 - y = 1/(1+e^z), both to full relative precision, and
  // log(y (1 - y)) = -|z| - 2 log(1 + e^-|z|)
  const float t = __expf(-fabsf(z));
  const float r = 1.f / (1.f + t);
  y = z >= 0.f ? r : t * r;
  yc = z >= 0.f ? t * r : r;
  lsp = -fabsf(z) - 2.f * log1pf(t);
}

// CTA prologue / epilogue of the sampling kernels: the MMA-completion barrier
// and the tensor-memory allocation (warp 0), released on every exit path.
template <class PH>
__device__ inline uint32_t flow_tc_begin(FlowSampSmem<PH>& S) {
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&S.mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    S.abort = 0;
  }
  if (threadIdx.x < 32) {
    tmem_alloc(smem_u32(&S.tmem), F_TMEM_COLS);
    tmem_relinquish();
  }
  // columns 128-143 of the activation operand are constant: 1, 1, 0, ..., 0
  // (they multiply the two parts of the hidden bias)
  for (int r = threadIdx.x; r < FROWS; r += blockDim.x) {
    const uint32_t one = pack_bf16(1.f, 1.f);
    *reinterpret_cast<uint4*>(&S.Act[umma_kmajor(r, FH, FKH)]) = make_uint4(one, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(&S.Act[umma_kmajor(r, FH + 8, FKH)]) = make_uint4(0u, 0u, 0u, 0u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return S.tmem;
}

template <class PH>
__device__ inline void flow_tc_end(FlowSampSmem<PH>& S, uint32_t tmem) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, F_TMEM_COLS);
  }
}

// Layer k's operands into shared memory (B operands copied as laid out in
// global memory), with the per-item bias c W1c + b1 folded into K 12-13 of the
// first layer's operand (the input carries 1, 1 there).
template <class PH>
__device__ inline void flow_tc_load_layer(FlowSampSmem<PH>& S, const FlowW* __restrict__ W,
                                          const FlowB* __restrict__ Bw, int k) {
  // asynchronous 16-byte copies (all in flight at once), completed below
  const uint4* s2 = reinterpret_cast<const uint4*>(&Bw->W2u[k][0]);
  uint4* d2 = reinterpret_cast<uint4*>(S.W2u);
  for (int t = threadIdx.x; t < FH * FKH / 8; t += blockDim.x) cp_async16(&d2[t], &s2[t]);
  const uint4* s1 = reinterpret_cast<const uint4*>(&Bw->W1u[k][0]);
  uint4* d1 = reinterpret_cast<uint4*>(S.W1u);
  for (int t = threadIdx.x; t < (int)(sizeof(S.W1u) / 16); t += blockDim.x) cp_async16(&d1[t], &s1[t]);
  const uint4* s3 = reinterpret_cast<const uint4*>(&Bw->W3t[k][0][0]);
  uint4* d3 = reinterpret_cast<uint4*>(&S.W3t[0][0]);
  for (int t = threadIdx.x; t < (int)(sizeof(S.W3t) / 16); t += blockDim.x) cp_async16(&d3[t], &s3[t]);
  float cb[(FH + THREADS - 1) / THREADS];
#pragma unroll
  for (int i = 0; i < (FH + THREADS - 1) / THREADS; ++i) {
    const int n = threadIdx.x + i * THREADS;
    if (n < FH) {
      float v = W->b1[k][n];
#pragma unroll
      for (int q = 0; q < FC; ++q) v = fmaf(S.c[q], W->W1c[k][q][n], v);
      cb[i] = v;
    }
  }
  cp_async_wait_all();
  __syncthreads();   // W1u copied: its K 12-13 now take the item's bias c W1c + b1 (split)
#pragma unroll
  for (int i = 0; i < (FH + THREADS - 1) / THREADS; ++i) {
    const int n = threadIdx.x + i * THREADS;
    if (n < FH) {
      const float hi = bf16_hi(cb[i]);
      S.W1u[umma_kmajor(n, 12, 16)] = __float2bfloat16_rn(hi);
      S.W1u[umma_kmajor(n, 13, 16)] = __float2bfloat16_rn(cb[i] - hi);
    }
  }
  if (threadIdx.x < 16) S.b3[threadIdx.x] = threadIdx.x < 8 ? W->b3[k][threadIdx.x] : 0.f;
}

// Accumulator columns 64 (warp / 4) .. + 63 of this warp's 32 rows (tensor-memory
// lanes 32 (warp % 4) ..) -> ReLU + BF16 -> the same columns and rows of Act, the
// operand of the next product (the biases are folded into the products).
template <class PH>
__device__ inline void flow_tc_epilogue(FlowSampSmem<PH>& S, uint32_t taddr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, row = 32 * q + lane;
  const int cbase = 64 * (warp >> 2);
  float v[64];
  tmem_ld64(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)cbase, v);
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int col0 = cbase + 8 * cc;
    uint32_t pk[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) pk[i] = pack_bf16_relu(v[8 * cc + 2 * i], v[8 * cc + 2 * i + 1]);
    *reinterpret_cast<uint4*>(&S.Act[umma_kmajor(row, col0, FKH)]) =
        make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// Thread pair (row, half) with row = thread % 128: K 0-7 (half 0) or K 8-15
// (half 1) of the first layer's input row of coupling layer k,
// z_A (at zr, stride 8) in the two-part BF16 split [hi | lo | hi | 1 1 0 0] that
// the split weights [W1a hi | W1a hi | W1a lo | bias hi, bias lo, 0 0] turn into
// z W1a + c W1c + b1 to ~16 bits.
template <class PH>
__device__ inline void flow_tc_first_operand(FlowSampSmem<PH>& S, int k, int row, int half,
                                             const float* zr) {
  const int na = flow_na(k);
  float zh[4], zl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float z = j < na ? zr[flow_a(k, j)] : 0.f;
    zh[j] = bf16_hi(z);
    zl[j] = z - zh[j];
  }
  const uint32_t h01 = pack_bf16(zh[0], zh[1]), h23 = pack_bf16(zh[2], zh[3]);
  if (half == 0)
    *reinterpret_cast<uint4*>(&S.A1[umma_kmajor(row, 0, 16)]) =
        make_uint4(h01, h23, pack_bf16(zl[0], zl[1]), pack_bf16(zl[2], zl[3]));
  else
    *reinterpret_cast<uint4*>(&S.A1[umma_kmajor(row, 8, 16)]) =
        make_uint4(h01, h23, pack_bf16(1.f, 1.f), 0u);
}

// One tcgen05 product D[tmem] = A B^T over n_k K-steps of 16, both operands
// K-major in shared memory (row strides sbo_a, sbo_b bytes), issued by thread 0,
// which waits for its completion; every thread then passes a barrier. False if
// the wait gave up (S.abort is then set for the CTA).
__device__ __forceinline__ bool flow_tc_mma(uint32_t d_tmem, uint32_t a_addr, uint32_t sbo_a,
                                            uint32_t b_addr, uint32_t sbo_b, int n_k,
                                            uint32_t idesc, uint32_t mbar, uint32_t& phase,
                                            int* abort) {
  fence_async_smem();   // generic-proxy operand writes -> the tensor core
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    for (int s = 0; s < n_k; ++s)
      umma_bf16(d_tmem, umma_desc(a_addr + 256u * (uint32_t)s, 128, sbo_a),
                umma_desc(b_addr + 256u * (uint32_t)s, 128, sbo_b), idesc, s > 0 ? 1u : 0u);
    umma_commit(mbar);
    if (!mbar_wait(mbar, phase, c_tc_wait_limit)) {
      // give up, but first drain the committed products (bounded as well) so that
      // nothing writes this CTA's tensor memory after it is released
      *abort = 1;
      mbar_wait(mbar, phase, F_DRAIN_LIMIT);
    }
  }
  phase ^= 1u;
  __syncthreads();   // the issuing thread saw the product complete
  tc_fence_after();
  return *abort == 0;
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr));
}

// One warp, output layer of coupling layer k for tile rows rl .. rl + 15: the
// hidden activations come from Act (each 8 x 8 core matrix of the UMMA layout
// is one ldmatrix tile), (s_raw | t) = h2 W3 + b3 by mma.sync, then the affine
// update of the z rows at zr and their log-Jacobian.
template <class PH>
__device__ inline void flow_output_layer(FlowSampSmem<PH>& S, int k, int rl, float* zr) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t base = smem_u32(S.Act);
  const int lrow = rl + (lane & 7) + ((lane >> 3) & 1) * 8, lcol = (lane >> 4) * 8;
  // two independent accumulation chains (even and odd K steps) halve the
  // dependent mma.sync latency
  float o[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  const __nv_bfloat16* brow = &S.W3t[g][0];
#pragma unroll
  for (int kk = 0; kk < FH / 16; ++kk) {
    uint32_t a[4];
    ldmatrix_x4(a, base + 2u * (uint32_t)umma_kmajor(lrow, 16 * kk + lcol, FKH));
    mma_bf16(o[kk & 1], a, *reinterpret_cast<const uint32_t*>(brow + 16 * kk + 2 * t),
             *reinterpret_cast<const uint32_t*>(brow + 16 * kk + 2 * t + 8));
  }
  const float bo0 = S.b3[2 * t], bo1 = S.b3[2 * t + 1];
  const float v0 = o[0][0] + o[1][0] + bo0, v1 = o[0][1] + o[1][1] + bo1;
  const float v2 = o[0][2] + o[1][2] + bo0, v3 = o[0][3] + o[1][3] + bo1;
  float v[8];
#pragma unroll
  for (int src = 0; src < 4; ++src) {
    const int sl = (lane & ~3) | src;
    const float x0 = __shfl_sync(0xffffffffu, v0, sl), x1 = __shfl_sync(0xffffffffu, v1, sl);
    const float x2 = __shfl_sync(0xffffffffu, v2, sl), x3 = __shfl_sync(0xffffffffu, v3, sl);
    v[2 * src] = t == 1 ? x2 : x0;
    v[2 * src + 1] = t == 1 ? x3 : x1;
  }
  if (t < 2) {
    float* row = zr + (g + 8 * t) * 8;
    if (k & 1) flow_update_row<FD / 2 + 1>(row, v, k);
    else flow_update_row<FD / 2>(row, v, k);
  }
}

// One pass of a CTA over points q0 .. q0 + nrow of an item (nrow a multiple of
// FROWS, at most FCH; rows at or past p1 are computed but not used): base draw,
// the coupling layers, then out(r, y, yc, log|dy/du|) per used row, threads
// striding over rows. Per 128-row tile and layer, two tcgen05 products: the
// first layer (K 16: split BF16 input and the item bias) and the hidden layer
// (K 144, bias folded in), each followed by a tensor-memory epilogue (ReLU, BF16
// repack into Act); then the output layer (N 8) per warp on mma.sync from Act and
// the affine update of the z rows. False if an MMA-completion wait gave up (the
// CTA then stops issuing work).
template <class PH, class Out>
__device__ inline bool flow_pass(FlowSampSmem<PH>& S, uint32_t tmem, uint32_t& phase,
                                 const FlowW* __restrict__ W, const FlowB* __restrict__ Bw,
                                 const PhiloxKey& key, uint32_t eid, int perm, uint32_t idx_base,
                                 uint32_t q0, uint32_t nrow, uint32_t p1, Out& out) {
  constexpr int D = PH::D;
  static_assert(D == FD, "the flow is built for the 7-dimensional ttbar integral");
  static_assert(THREADS == 2 * FROWS, "two threads build each row of the first-layer input");
  constexpr uint32_t ID_H = umma_idesc_bf16(FROWS, FH);
  for (uint32_t r = threadIdx.x; r < nrow; r += THREADS) {
    const uint32_t p = q0 + r;
    float u[D];
    if (p < p1) {
      point_uniforms<D>(key, eid, (uint32_t)perm, idx_base + p, u, TAG_FLOW);
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) u[j] = 0.5f;
    }
    float lj = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float z = __logf(u[j]) - log1pf(-u[j]);
      S.zs[r * 8 + j] = z;
      lj -= log_sig_prime(z);
    }
    S.zs[r * 8 + 7] = lj;
  }
  const uint32_t act = smem_u32(S.Act), a1 = smem_u32(S.A1), w1 = smem_u32(S.W1u);
  const uint32_t w2 = smem_u32(S.W2u), mbar = smem_u32(&S.mbar);
  const int warp = threadIdx.x >> 5;
  for (int k = 0; k < FK; ++k) {
    // the previous layer's products are complete and its z updates visible
    tc_fence_before();
    __syncthreads();
    if (S.abort) return false;
    flow_tc_load_layer(S, W, Bw, k);
    const int frow = threadIdx.x & (FROWS - 1), fhalf = threadIdx.x / FROWS;
    flow_tc_first_operand(S, k, frow, fhalf, &S.zs[frow * 8]);
    for (uint32_t t0 = 0; t0 < nrow; t0 += FROWS) {
      // first layer (item bias folded into K 12-13), ReLU -> Act. The barrier in
      // flow_tc_mma also orders the previous tile's output layer (reads of Act)
      // before this tile's epilogue writes Act.
      if (!flow_tc_mma(tmem, a1, 16 * 16, w1, 16 * 16, 1, ID_H, mbar, phase, &S.abort))
        return false;
      flow_tc_epilogue(S, tmem);
      // A1 is free (the product above is complete): the next tile's input, whose
      // z_A rows the current tile's update does not touch
      if (t0 + FROWS < nrow)
        flow_tc_first_operand(S, k, frow, fhalf, &S.zs[(t0 + FROWS + frow) * 8]);
      // hidden layer (bias folded into K 128-129), ReLU -> Act
      if (!flow_tc_mma(tmem, act, 16 * FKH, w2, 16 * FKH, FKH / 16, ID_H, mbar, phase, &S.abort))
        return false;
      flow_tc_epilogue(S, tmem);
      tc_fence_before();
      __syncthreads();   // Act holds the whole tile's hidden output
      // output layer per warp on mma.sync, then the affine update of its 16 rows
      flow_output_layer(S, k, 16 * warp, &S.zs[(t0 + 16 * warp) * 8]);
    }
  }
  __syncthreads();
  if (S.abort) return false;
  for (uint32_t r = threadIdx.x; r < nrow; r += THREADS) {
    if (q0 + r >= p1) continue;
    float y[D], yc[D];
    float lj = S.zs[r * 8 + 7];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float lsp;
      sigmoid_pair(S.zs[r * 8 + j], y[j], yc[j], lsp);
      lj += lsp;
    }
    out(r, y, yc, lj);
  }
  __syncthreads();
  return true;
}

// Flow-sampled round of the adaptive integrator: persistent CTAs walk the
// compacted active list in tiles (as the VEGAS round kernel does) and write
// one compensated (sum w, sum w^2) slot per tile. With HIST, every point also
// adds w^2 to its item's histogram over NG uniform bins per dimension (hist,
// n_items x D x NG), the importance a VEGAS grid refinement starts from.
template <class PH, int MINB, bool HIST>
__global__ void __launch_bounds__(THREADS, MINB)
k_flow_round_sample(const float* __restrict__ recs, ProcConst P,
                    const __grid_constant__ PhiloxKey key,
                    uint64_t event_id_base, const int32_t* __restrict__ active,
                    const RoundCtl* __restrict__ ctl, uint32_t idx_base, uint32_t pts_item,
                    const FlowW* __restrict__ W, const FlowB* __restrict__ Bw,
                    const typename PH::Cache* __restrict__ caches,
                    const float* __restrict__ feats, Slot* __restrict__ slots,
                    float* __restrict__ hist, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char flow_smem[];
  FlowSampSmem<PH>& S = *reinterpret_cast<FlowSampSmem<PH>*>(flow_smem);
  const uint32_t tmem = flow_tc_begin(S);
  uint32_t phase = 0;
  bool alive = true;
  const int n_act = ctl->n_active, tpi = ctl->tiles_per_item;
  const int64_t n_tiles = (int64_t)n_act * tpi;
  const uint32_t per_tile = ((pts_item + tpi - 1) / tpi + FROWS - 1) / FROWS * FROWS;
  for (int64_t tile = blockIdx.x; tile < n_tiles && alive; tile += gridDim.x) {
    const int32_t item = active[tile / tpi];
    const uint32_t k = (uint32_t)(tile % tpi);
    const int64_t ev = item / PH::NPERM;
    const int perm = (int)(item % PH::NPERM);
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(caches + item);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&S.cache);
      for (int t = threadIdx.x; t < (int)(sizeof(typename PH::Cache) / 4); t += blockDim.x)
        dst[t] = src[t];
      if (threadIdx.x < FC) S.c[threadIdx.x] = feats[(int64_t)item * FC + threadIdx.x];
      if (HIST)
        for (int t = threadIdx.x; t < PH::D * NG; t += blockDim.x) S.hist[t] = 0.f;
    }
    __syncthreads();
    const uint32_t eid = (uint32_t)(event_id_base + (uint64_t)ev);
    const uint32_t p0 = min(k * per_tile, pts_item);
    const uint32_t p1 = min(p0 + per_tile, pts_item);
    Kahan32 a1, a2;
    uint32_t nbad = 0;
    if (S.cache.ok) {
      auto acc = [&](uint32_t, const float (&y)[PH::D], const float (&yc)[PH::D], float lj) {
        const float w = PH::eval(S.cache, P, y, yc) * __expf(lj);
        if (isfinite(w)) {
          a1.add(w);
          a2.add(w * w);
          if (HIST) {
#pragma unroll
            for (int j = 0; j < PH::D; ++j) {
              const int b = min((int)(y[j] * (float)NG), NG - 1);
              atomicAdd(&S.hist[j * NG + b], w * w);
            }
          }
        } else {
          ++nbad;
        }
      };
#pragma unroll 1
      for (uint32_t q0 = p0; q0 < p1; q0 += FCH) {
        const uint32_t nrow = min((uint32_t)FCH, (p1 - q0 + FROWS - 1) / FROWS * FROWS);
        if (!flow_pass<PH>(S, tmem, phase, W, Bw, key, eid, perm, idx_base, q0, nrow, p1, acc)) {
          alive = false;
          break;
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
    if (HIST) {
      float* hg = hist + (int64_t)item * (PH::D * NG);
      for (int t = threadIdx.x; t < PH::D * NG; t += blockDim.x)
        if (S.hist[t] != 0.f) atomicAdd(&hg[t], S.hist[t]);
    }
    __syncthreads();
  }
  if (!alive && threadIdx.x == 0) atomicExch(err, 1);
  flow_tc_end(S, tmem);
}

// Flow-sampled points of one item, one output row per point (parity tests):
// final logits z (y = sigmoid z), log|dy/du| and the weight with its
// prefactor. CTA b handles points b FCH .. of the n requested.
template <class PH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
k_flow_points(const float* __restrict__ rec, int perm, ProcConst P, TFConst T,
              const __grid_constant__ PhiloxKey key,
              uint32_t event_id, uint32_t point0, uint32_t n, const FlowW* __restrict__ W,
              const FlowB* __restrict__ Bw, float* __restrict__ z_out, float* __restrict__ lj_out,
              double* __restrict__ w_out, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char flow_smem[];
  FlowSampSmem<PH>& S = *reinterpret_cast<FlowSampSmem<PH>*>(flow_smem);
  const uint32_t tmem = flow_tc_begin(S);
  uint32_t phase = 0;
  if (threadIdx.x == 0) PH::setup(rec, perm, P, T, S.cache);
  if (threadIdx.x == 32) flow_features(rec, perm, S.c);
  __syncthreads();
  const uint32_t q0 = blockIdx.x * FCH;
  const uint32_t nrow = min((uint32_t)FCH, (n - q0 + FROWS - 1) / FROWS * FROWS);
  auto put = [&](uint32_t r, const float (&y)[PH::D], const float (&yc)[PH::D], float lj) {
    const uint32_t i = q0 + r;
    const float w = S.cache.ok ? PH::eval(S.cache, P, y, yc) * __expf(lj) : 0.f;
#pragma unroll
    for (int j = 0; j < PH::D; ++j) z_out[(size_t)i * PH::D + j] = S.zs[r * 8 + j];
    lj_out[i] = lj;
    w_out[i] = (double)w * P.prefactor;
  };
  if (!flow_pass<PH>(S, tmem, phase, W, Bw, key, event_id, perm, point0 + q0, 0, nrow, n - q0,
                     put) &&
      threadIdx.x == 0)
    atomicExch(err, 1);
  flow_tc_end(S, tmem);
}

}  // namespace mem
