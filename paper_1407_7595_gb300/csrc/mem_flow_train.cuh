// Training of the learned importance sampler on VEGAS-weighted samples:
// loss L = sum_i w_i log|dy/du|(y_i) (= -sum_i w_i log q(y_i), w normalised per
// item: the KL divergence from the integrand's normalised density to q),
// evaluated through the inverse map and differentiated by hand-written reverse
// mode. One CTA = 128 samples of one item (one conditioning vector).
//
// Every 128 x 128 contraction runs on the fifth-generation tensor cores
// (tcgen05.mma kind::f16, BF16 operands in shared memory in the canonical
// K-major layout, FP32 accumulators in tensor memory, one issuing thread, one
// mbarrier commit per group of products):
//   inverse and backward passes, per layer: a2 = relu(a1) W2 + b2 (bias folded
//     into the operand, as in the sampling kernels);
//   backward, per layer: dW2 = relu(a1)^T dL/da2, dL/dh1 = dL/da2 W2^T and
//     dW3 = relu(a2)^T dL/d(out) (N 16, 8 used).
// The |A|-wide first layer, the 8-wide output layer and the reductions over
// samples run in FP32 on the CUDA cores. Tensor memory: 512 columns (a2 | dW2 |
// dL/dh1 | dW3), so one CTA per SM (its shared memory alone ensures that).
// Weight gradients are reduced across CTAs with FP32 atomics into a FlowW-shaped
// buffer. Every completion wait is bounded; a CTA whose wait gives up drains
// its products, releases tensor memory and raises the error flag.
#pragma once
#include "mem_flow.cuh"
#include "mem_umma.cuh"

namespace mem {

constexpr int TS = 128;                      // samples per CTA
constexpr uint32_t FT_TMEM_COLS = 512;
constexpr uint32_t FT_COL_A2 = 0, FT_COL_DW2 = 128, FT_COL_GH1 = 256, FT_COL_DW3 = 384;
constexpr uint32_t FT_DRAIN_LIMIT = 1u << 22;
// Poll limit of the training kernel's MMA-completion waits (mem_set_tc_wait_limit).
__constant__ uint32_t c_train_wait_limit = 1u << 20;

struct __align__(1024) FlowTrainSmem {
  __nv_bfloat16 act[FH * FKH];   // [s][k], K 144: relu(a1) | 1 1 0 ...; then relu(a2)^T [h][s], K 128
  __nv_bfloat16 h1t[FH * TS];    // relu(a1)^T [in][s]; then FP32 staging of dL/da1 columns 0-63
  __nv_bfloat16 ga2[TS * FH];    // dL/da2 [s][out]
  __nv_bfloat16 ga2t[FH * TS];   // dL/da2^T [out][s]; then FP32 staging of dL/da1 columns 64-127
  __nv_bfloat16 wb[FH * FKH];    // B operand: W2u (N 128 x K 144) or W2v (N 128 x K 128)
  __nv_bfloat16 got[16 * TS];    // dL/d(out)^T [o][s], rows 2|B| .. 15 zero
  float W1a[4][FH];
  float cb1[FH];                 // c W1c + b1 of the CTA's item
  float W3f[FH][8];              // the BF16 output weights [in][out] as FP32
  float b3[8];
  float zc[TS][8];               // z of the current level
  float so[FK][TS][8];           // raw MLP outputs (s_raw | t) of every layer
  float gz[TS][8];               // dL/dz of the current level
  float gof[TS][8];              // dL/d(out) (BF16-rounded); partial sums between column halves
  float part[2][5][FH];          // per column, two row halves: sum dL/da1, sum z_A dL/da1 (4)
  float c[FC];
  float w[TS];
  unsigned long long mbar;
  uint32_t tmem;
  int abort;
};

// One product D[tmem] (+)= A B^T over n_k K-steps of 16 (both operands K-major,
// SBO = 16 K bytes), issued by the calling thread.
__device__ __forceinline__ void ft_mma(uint32_t d_tmem, uint32_t a_addr, uint32_t sbo_a,
                                       uint32_t b_addr, uint32_t sbo_b, int n_k, uint32_t idesc) {
  for (int s = 0; s < n_k; ++s)
    umma_bf16(d_tmem, umma_desc(a_addr + 256u * (uint32_t)s, 128, sbo_a),
              umma_desc(b_addr + 256u * (uint32_t)s, 128, sbo_b), idesc, s > 0 ? 1u : 0u);
}

// Every thread: publish its shared-memory operand writes to the tensor core; thread
// 0 issues the products (issue()), commits them to the mbarrier and waits (bounded;
// after a give-up it drains them with a second bounded wait); every thread then
// passes a barrier. False when the wait gave up (S.abort is set for the CTA).
template <class F>
__device__ __forceinline__ bool ft_products(FlowTrainSmem& S, uint32_t& phase, F issue) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    issue();
    const uint32_t mbar = smem_u32(&S.mbar);
    umma_commit(mbar);
    if (!mbar_wait(mbar, phase, c_train_wait_limit)) {
      S.abort = 1;
      mbar_wait(mbar, phase, FT_DRAIN_LIMIT);
    }
  }
  phase ^= 1u;
  __syncthreads();
  tc_fence_after();
  return S.abort == 0;
}

// The B operand of the hidden products: W2u (with the bias folded) or W2v.
__device__ inline void ft_load_wb(FlowTrainSmem& S, const FlowB* __restrict__ Bw, int k, bool w2v) {
  const uint4* src = w2v ? reinterpret_cast<const uint4*>(&Bw->W2v[k][0])
                         : reinterpret_cast<const uint4*>(&Bw->W2u[k][0]);
  const int n16 = w2v ? FH * FH / 8 : FH * FKH / 8;
  uint4* dst = reinterpret_cast<uint4*>(S.wb);
  for (int t = threadIdx.x; t < n16; t += blockDim.x) cp_async16(&dst[t], &src[t]);
  cp_async_wait_all();
  __syncthreads();
}

// The FP32 parts of layer k: W1a, c W1c + b1, the BF16 output weights, b3.
__device__ inline void ft_load_small(FlowTrainSmem& S, const FlowW* __restrict__ W,
                                     const FlowB* __restrict__ Bw, int k) {
  for (int t = threadIdx.x; t < 4 * FH; t += blockDim.x) (&S.W1a[0][0])[t] = (&W->W1a[k][0][0])[t];
  for (int n = threadIdx.x; n < FH; n += blockDim.x) {
    float v = W->b1[k][n];
#pragma unroll
    for (int q = 0; q < FC; ++q) v = fmaf(S.c[q], W->W1c[k][q][n], v);
    S.cb1[n] = v;
  }
  for (int t = threadIdx.x; t < FH * 8; t += blockDim.x) {
    const int i = t >> 3, o = t & 7;
    S.W3f[i][o] = __bfloat162float(Bw->W3t[k][o][i]);
  }
  if (threadIdx.x < 8) S.b3[threadIdx.x] = W->b3[k][threadIdx.x];
}

// First layer of layer k for this thread's sample `row` and columns 64 half ..:
// relu(c W1c + b1 + z_A W1a) in FP32, BF16 into act (and, for the backward pass,
// transposed into h1t); half 0 also writes the bias columns 128-143 (1, 1, 0 ...).
__device__ inline void ft_first_layer(FlowTrainSmem& S, int k, int row, int half, bool transposed) {
  const int na = flow_na(k);
  float za[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) za[j] = j < na ? S.zc[row][flow_a(k, j)] : 0.f;
#pragma unroll 2
  for (int cc = 0; cc < 8; ++cc) {
    const int n0 = 64 * half + 8 * cc;
    uint32_t pk[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int n = n0 + 2 * i + h;
        float a = S.cb1[n];
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fmaf(za[j], S.W1a[j][n], a);
        v[h] = a;
      }
      pk[i] = pack_bf16_relu(v[0], v[1]);
    }
    *reinterpret_cast<uint4*>(&S.act[umma_kmajor(row, n0, FKH)]) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    if (transposed) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&pk[i]);
        S.h1t[umma_kmajor(n0 + 2 * i, row, TS)] = b.x;
        S.h1t[umma_kmajor(n0 + 2 * i + 1, row, TS)] = b.y;
      }
    }
  }
  if (half == 0) {
    *reinterpret_cast<uint4*>(&S.act[umma_kmajor(row, FH, FKH)]) =
        make_uint4(pack_bf16(1.f, 1.f), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(&S.act[umma_kmajor(row, FH + 8, FKH)]) = make_uint4(0u, 0u, 0u, 0u);
  }
}

__device__ __forceinline__ uint32_t ft_lane_base(uint32_t tmem) {
  const int warp = threadIdx.x >> 5;
  return tmem + ((uint32_t)(32 * (warp & 3)) << 16);
}

// One training CTA: samples y (TS x 7), weights w (TS), conditioning c (16) of item
// batch[blockIdx.x]; zscr: (FK + 1) x TS x 8 floats per CTA (z of every level).
__global__ void __launch_bounds__(256, 1)
k_flow_train(const FlowW* __restrict__ W, const FlowB* __restrict__ Bw,
             const float* __restrict__ ys, const float* __restrict__ ws,
             const float* __restrict__ cs, const int32_t* __restrict__ batch,
             FlowW* __restrict__ G, float* __restrict__ loss_out, float* __restrict__ zscr,
             int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char raw[];
  FlowTrainSmem& S = *reinterpret_cast<FlowTrainSmem*>(raw);
  const int item = batch[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane;   // tensor-memory lane = sample (or hidden) row
  const int half = warp >> 2;               // accumulator columns 64 half .. + 63
  float* Z = zscr + (size_t)blockIdx.x * (FK + 1) * TS * 8;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&S.mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    S.abort = 0;
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(&S.tmem), FT_TMEM_COLS);
    tmem_relinquish();
  }
  if (threadIdx.x < FC) S.c[threadIdx.x] = cs[(int64_t)item * FC + threadIdx.x];
  for (int p = threadIdx.x; p < TS; p += blockDim.x) {
    S.w[p] = ws[(int64_t)item * TS + p];
    for (int j = 0; j < 8; ++j) {
      float z = 0.f;
      if (j < FD) {
        const float y = ys[((int64_t)item * TS + p) * FD + j];
        z = logf(y) - log1pf(-y);
      }
      S.zc[p][j] = z;
      Z[((size_t)FK * TS + p) * 8 + j] = z;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t tl = ft_lane_base(tmem);
  constexpr uint32_t ID_N128 = umma_idesc_bf16(128, 128), ID_N16 = umma_idesc_bf16(128, 16);
  const uint32_t a_act = smem_u32(S.act), a_h1t = smem_u32(S.h1t), a_ga2 = smem_u32(S.ga2);
  const uint32_t a_ga2t = smem_u32(S.ga2t), a_wb = smem_u32(S.wb), a_got = smem_u32(S.got);
  uint32_t phase = 0;
  bool ok = true;

  // ---- inverse pass: z_K -> z_0, keeping the raw outputs of every layer
  for (int k = FK - 1; k >= 0 && ok; --k) {
    ft_load_small(S, W, Bw, k);
    ft_load_wb(S, Bw, k, false);
    ft_first_layer(S, k, row, half, false);
    ok = ft_products(S, phase, [&] { ft_mma(tmem + FT_COL_A2, a_act, 16 * FKH, a_wb, 16 * FKH, FKH / 16, ID_N128); });
    if (!ok) break;
    // output layer from the BF16 hidden activations, this thread's 64 columns
    float v[64];
    tmem_ld64(tl + FT_COL_A2 + 64 * half, v);
    float o[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      const float h = __bfloat162float(__float2bfloat16_rn(fmaxf(v[i], 0.f)));
#pragma unroll
      for (int j = 0; j < 8; ++j) o[j] = fmaf(h, S.W3f[64 * half + i][j], o[j]);
    }
    if (half == 1)
#pragma unroll
      for (int j = 0; j < 8; ++j) S.gof[row][j] = o[j];
    tc_fence_before();
    __syncthreads();
    if (half == 0) {
      const int nb = flow_nb(k);
#pragma unroll
      for (int j = 0; j < 8; ++j) S.so[k][row][j] = o[j] + S.gof[row][j] + S.b3[j];
      for (int j = 0; j < nb; ++j) {
        const float s = F_SMAX * tanhf(S.so[k][row][j] * (1.f / F_SMAX));
        const int idx = flow_b(k, j);
        S.zc[row][idx] = (S.zc[row][idx] - S.so[k][row][nb + j]) * __expf(-s);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) Z[((size_t)k * TS + row) * 8 + j] = S.zc[row][j];
    }
    __syncthreads();
  }

  if (ok) {
    // ---- loss sum w log|dy/du| and dL/dz0 (the sum log sig'(z_K) term does not
    // depend on the parameters: it enters the loss value, not the gradient)
    float lsum = 0.f;
    for (int p = threadIdx.x; p < TS; p += blockDim.x) {
      float lp = 0.f;
      for (int k = 0; k < FK; ++k)
        for (int j = 0; j < flow_nb(k); ++j) lp += F_SMAX * tanhf(S.so[k][p][j] * (1.f / F_SMAX));
      for (int j = 0; j < 8; ++j) {
        float gzz = 0.f;
        if (j < FD) {
          const float z0 = S.zc[p][j];
          lp += log_sig_prime(Z[((size_t)FK * TS + p) * 8 + j]) - log_sig_prime(z0);
          const float sg = 1.f / (1.f + __expf(-z0));
          gzz = -S.w[p] * (1.f - 2.f * sg);
        }
        S.gz[p][j] = gzz;
      }
      lsum += S.w[p] * lp;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(loss_out, lsum);
    __syncthreads();
  }

  // ---- backward, layer 0 upwards
  for (int k = 0; k < FK && ok; ++k) {
    const int na = flow_na(k), nb = flow_nb(k);
    ft_load_small(S, W, Bw, k);
    for (int t = threadIdx.x; t < TS * 8; t += blockDim.x) S.zc[t >> 3][t & 7] = Z[(size_t)(k + 1) * TS * 8 + t];
    ft_load_wb(S, Bw, k, false);   // (its barrier also publishes zc and the small parts)
    // output gradient g_o = (dL/ds_raw | dL/dt) per sample, dL/dz_{k+1}[B]
    for (int p = threadIdx.x; p < TS; p += blockDim.x) {
      float go[16];
#pragma unroll
      for (int o = 0; o < 16; ++o) go[o] = 0.f;
      for (int j = 0; j < nb; ++j) {
        const int idx = flow_b(k, j);
        const float th = tanhf(S.so[k][p][j] * (1.f / F_SMAX));
        const float s = F_SMAX * th;
        const float tt = S.so[k][p][nb + j];
        const float e = __expf(-s);
        const float gzb = S.gz[p][idx];
        const float g_t = -gzb * e;
        const float g_s = -gzb * (S.zc[p][idx] - tt) * e + S.w[p];
        go[j] = g_s * (1.f - th * th);
        go[nb + j] = g_t;
        S.gz[p][idx] = gzb * e;   // dL/dz_{k+1}[B]; [A] keeps the pass-through
      }
#pragma unroll
      for (int o = 0; o < 16; ++o) {
        const __nv_bfloat16 b = __float2bfloat16_rn(go[o]);
        S.got[umma_kmajor(o, p, TS)] = b;
        if (o < 8) S.gof[p][o] = __bfloat162float(b);
      }
    }
    ft_first_layer(S, k, row, half, true);
    __syncthreads();   // gof complete
    if (threadIdx.x < 8) {
      float s3 = 0.f;
      for (int p = 0; p < TS; ++p) s3 += S.gof[p][threadIdx.x];
      atomicAdd(&G->b3[k][threadIdx.x], s3);
    }
    // a2 = relu(a1) W2 + b2 (recomputed)
    ok = ft_products(S, phase, [&] { ft_mma(tmem + FT_COL_A2, a_act, 16 * FKH, a_wb, 16 * FKH, FKH / 16, ID_N128); });
    if (!ok) break;
    {
      float v[64];
      tmem_ld64(tl + FT_COL_A2 + 64 * half, v);
      float go[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) go[o] = S.gof[row][o];
#pragma unroll 2
      for (int cc = 0; cc < 8; ++cc) {
        const int n0 = 64 * half + 8 * cc;
        uint32_t pk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float g2[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int n = n0 + 2 * i + h;
            const float a2 = v[8 * cc + 2 * i + h];
            // relu(a2)^T as the A operand of dW3 (the act buffer is free: the product is done)
            S.act[umma_kmajor(n, row, TS)] = __float2bfloat16_rn(fmaxf(a2, 0.f));
            float gg = 0.f;
#pragma unroll
            for (int o = 0; o < 8; ++o) gg = fmaf(go[o], S.W3f[n][o], gg);
            g2[h] = a2 > 0.f ? gg : 0.f;
          }
          pk[i] = pack_bf16(g2[0], g2[1]);
          __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&pk[i]);
          S.ga2t[umma_kmajor(n0 + 2 * i, row, TS)] = b.x;
          S.ga2t[umma_kmajor(n0 + 2 * i + 1, row, TS)] = b.y;
        }
        *reinterpret_cast<uint4*>(&S.ga2[umma_kmajor(row, n0, FH)]) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    tc_fence_before();
    __syncthreads();   // ga2 complete; the hidden product is done, so wb may be replaced
    if (threadIdx.x < FH) {
      float s2 = 0.f;
      for (int p = 0; p < TS; ++p) s2 += __bfloat162float(S.ga2[umma_kmajor(p, threadIdx.x, FH)]);
      atomicAdd(&G->b2[k][threadIdx.x], s2);
    }
    ft_load_wb(S, Bw, k, true);
    // dW3 = relu(a2)^T g_o, dW2 = relu(a1)^T dL/da2, dL/dh1 = dL/da2 W2^T
    ok = ft_products(S, phase, [&] {
      ft_mma(tmem + FT_COL_DW3, a_act, 16 * TS, a_got, 16 * TS, TS / 16, ID_N16);
      ft_mma(tmem + FT_COL_DW2, a_h1t, 16 * TS, a_ga2t, 16 * TS, TS / 16, ID_N128);
      ft_mma(tmem + FT_COL_GH1, a_ga2, 16 * FH, a_wb, 16 * FH, FH / 16, ID_N128);
    });
    if (!ok) break;
    {
      if (half == 0) {
        float d3[8];
        tmem_ld8(tl + FT_COL_DW3, d3);
#pragma unroll
        for (int o = 0; o < 8; o += 4)
          atomicAdd(reinterpret_cast<float4*>(&G->W3[k][row][o]), make_float4(d3[o], d3[o + 1], d3[o + 2], d3[o + 3]));
      }
      float v[64];
      tmem_ld64(tl + FT_COL_DW2 + 64 * half, v);
      // 16-byte vector atomics: a quarter of the gradient atomics (rows are 512 B aligned)
#pragma unroll 4
      for (int i = 0; i < 64; i += 4)
        atomicAdd(reinterpret_cast<float4*>(&G->W2[k][row][64 * half + i]),
                  make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
      // dL/da1 = dL/dh1 [a1 > 0] for this thread's sample and columns; dL/dz_A partials
      tmem_ld64(tl + FT_COL_GH1 + 64 * half, v);
      float za[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) za[j] = j < na ? S.zc[row][flow_a(k, j)] : 0.f;
      float dz[4] = {0.f, 0.f, 0.f, 0.f};
      float* stage = reinterpret_cast<float*>(half == 0 ? S.h1t : S.ga2t);   // [row][64]
#pragma unroll 8
      for (int i = 0; i < 64; ++i) {
        const int n = 64 * half + i;
        float a1 = S.cb1[n];
#pragma unroll
        for (int j = 0; j < 4; ++j) a1 = fmaf(za[j], S.W1a[j][n], a1);
        const float g1 = a1 > 0.f ? v[i] : 0.f;
        stage[row * 64 + i] = g1;
#pragma unroll
        for (int j = 0; j < 4; ++j) dz[j] = fmaf(g1, S.W1a[j][n], dz[j]);
      }
      if (half == 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) S.gof[row][j] = dz[j];
      tc_fence_before();
      __syncthreads();
      if (half == 0)
        for (int j = 0; j < na; ++j) S.gz[row][flow_a(k, j)] += dz[j] + S.gof[row][j];
      // column sums over the samples: thread (column n, row half rh)
      {
        const int n = threadIdx.x & (FH - 1), rh = threadIdx.x >> 7;
        const float* st = reinterpret_cast<const float*>(n < 64 ? S.h1t : S.ga2t);
        const int cn = n & 63;
        float cs0 = 0.f, cz[4] = {0.f, 0.f, 0.f, 0.f};
        for (int p = 64 * rh; p < 64 * rh + 64; ++p) {
          const float g1 = st[p * 64 + cn];
          cs0 += g1;
#pragma unroll
          for (int j = 0; j < 4; ++j) cz[j] = fmaf(j < na ? S.zc[p][flow_a(k, j)] : 0.f, g1, cz[j]);
        }
        S.part[rh][0][n] = cs0;
#pragma unroll
        for (int j = 0; j < 4; ++j) S.part[rh][1 + j][n] = cz[j];
      }
      __syncthreads();
      if (threadIdx.x < FH) {
        const int n = threadIdx.x;
        const float csn = S.part[0][0][n] + S.part[1][0][n];
        atomicAdd(&G->b1[k][n], csn);
        for (int q = 0; q < FC; ++q) atomicAdd(&G->W1c[k][q][n], S.c[q] * csn);
        for (int j = 0; j < na; ++j) atomicAdd(&G->W1a[k][j][n], S.part[0][1 + j][n] + S.part[1][1 + j][n]);
      }
      __syncthreads();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, FT_TMEM_COLS);
  }
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

// Adam on every parameter (FlowW-shaped buffers), then the gradient is cleared.
__global__ void k_flow_adam(FlowW* __restrict__ W, FlowW* __restrict__ m, FlowW* __restrict__ v,
                            FlowW* __restrict__ G, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, float scale) {
  float* w = reinterpret_cast<float*>(W);
  float* mm = reinterpret_cast<float*>(m);
  float* vv = reinterpret_cast<float*>(v);
  float* gg = reinterpret_cast<float*>(G);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gr = gg[i] * scale;
    const float mi = b1 * mm[i] + (1.f - b1) * gr;
    const float vi = b2 * vv[i] + (1.f - b2) * gr * gr;
    mm[i] = mi;
    vv[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    gg[i] = 0.f;
  }
}

}  // namespace mem
