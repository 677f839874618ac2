// Training of the learned importance sampler on VEGAS-weighted samples:
// loss L = sum_i w_i log|dy/du|(y_i) (= -sum_i w_i log q(y_i), w normalised per
// item: the KL divergence from the integrand's normalised density to q),
// evaluated through the inverse map and differentiated by hand-written reverse
// mode. One CTA = 128 samples of one item (one conditioning vector); per layer
// the MLP is recomputed in the backward pass (no stored hidden activations).
// Tensor-core GEMMs (mma.sync m16n8k16 BF16 -> FP32): the hidden layer of the
// recomputation, dW2 = h1^T g_a2, g_h1 = g_a2 W2^T and dW3 = h2^T g_o; FP32 for
// the |A|- and 8-wide parts. Weight gradients are reduced across CTAs with FP32
// atomics into a FlowW-shaped buffer.
#pragma once
#include "mem_flow.cuh"

namespace mem {

constexpr int TS = 128;  // samples per CTA

struct __align__(16) FlowTrainSmem {
  FlowLayerSmem L;
  __nv_bfloat16 H1[TS][FLD];   // relu(a1), BF16
  __nv_bfloat16 H2[TS][FLD];   // relu(a2), BF16
  __nv_bfloat16 GA2[TS][FLD];  // dL/da2, BF16
  __nv_bfloat16 GOt[8][FLD];   // dL/d(out) transposed: [o][sample]
  float zsnap[FK + 1][TS][8];  // z entering each inverse layer (index k+1) and z0
  float so[FK][TS][8];         // raw MLP outputs (s_raw | t) of each layer
  float gz[TS][8];             // dL/dz of the current level
  float c[FC];
  float w[TS];
  float colsum[FH];            // sum over samples of dL/da1 (for b1, W1c)
  float red[8];
};

__device__ __forceinline__ uint32_t ld_pair_T(const __nv_bfloat16* base, int ld, int r, int c) {
  // elements base[r][c] and base[r+1][c] packed (low = row r)
  const unsigned short lo = *reinterpret_cast<const unsigned short*>(base + r * ld + c);
  const unsigned short hi = *reinterpret_cast<const unsigned short*>(base + (r + 1) * ld + c);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Recompute the MLP of layer k for the warp's 16 rows from z (zin, row stride 8):
// stores relu(a1) to H1, relu(a2) to H2 (BF16) and returns nothing else.
__device__ inline void flow_train_recompute(FlowTrainSmem& S, int k, const float (*zin)[8], int r0) {
  const FlowLayerSmem& L = S.L;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int na = flow_na(k);
  float za0[4], za1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    za0[j] = j < na ? zin[r0 + g][flow_a(k, j)] : 0.f;
    za1[j] = j < na ? zin[r0 + g + 8][flow_a(k, j)] : 0.f;
  }
  uint32_t a[8][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    float h[2][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = kk * 16 + 2 * t + (q & 1) + ((q >> 1) << 3);
      float v0 = L.cb1[col], v1 = L.cb1[col];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v0 = fmaf(za0[j], L.W1a[j][col], v0);
        v1 = fmaf(za1[j], L.W1a[j][col], v1);
      }
      h[0][q] = fmaxf(v0, 0.f);
      h[1][q] = fmaxf(v1, 0.f);
    }
    a[kk][0] = pack_bf16(h[0][0], h[0][1]);
    a[kk][1] = pack_bf16(h[1][0], h[1][1]);
    a[kk][2] = pack_bf16(h[0][2], h[0][3]);
    a[kk][3] = pack_bf16(h[1][2], h[1][3]);
    const int c0 = kk * 16 + 2 * t;
    *reinterpret_cast<uint32_t*>(&S.H1[r0 + g][c0]) = a[kk][0];
    *reinterpret_cast<uint32_t*>(&S.H1[r0 + g + 8][c0]) = a[kk][1];
    *reinterpret_cast<uint32_t*>(&S.H1[r0 + g][c0 + 8]) = a[kk][2];
    *reinterpret_cast<uint32_t*>(&S.H1[r0 + g + 8][c0 + 8]) = a[kk][3];
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* brow = &L.W2t[j * 8 + g][0];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(brow + kk * 16 + 2 * t);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(brow + kk * 16 + 2 * t + 8);
      mma_bf16(acc, a[kk], b0, b1);
    }
    const int c0 = j * 8 + 2 * t;
    const float bb0 = L.b2[c0], bb1 = L.b2[c0 + 1];
    *reinterpret_cast<uint32_t*>(&S.H2[r0 + g][c0]) =
        pack_bf16(fmaxf(acc[0] + bb0, 0.f), fmaxf(acc[1] + bb1, 0.f));
    *reinterpret_cast<uint32_t*>(&S.H2[r0 + g + 8][c0]) =
        pack_bf16(fmaxf(acc[2] + bb0, 0.f), fmaxf(acc[3] + bb1, 0.f));
  }
}

// One training CTA: samples y (TS x 7), weights w (TS), conditioning c (16).
__global__ void __launch_bounds__(256, 1)
k_flow_train(const FlowW* __restrict__ W, const FlowB* __restrict__ Bw,
             const float* __restrict__ ys, const float* __restrict__ ws,
             const float* __restrict__ cs, const int32_t* __restrict__ batch,
             FlowW* __restrict__ G, float* __restrict__ loss_out) {
  extern __shared__ __align__(16) unsigned char raw[];
  FlowTrainSmem& S = *reinterpret_cast<FlowTrainSmem*>(raw);
  const int item = batch[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  if (threadIdx.x < FC) S.c[threadIdx.x] = cs[(int64_t)item * FC + threadIdx.x];
  for (int p = threadIdx.x; p < TS; p += blockDim.x) {
    S.w[p] = ws[(int64_t)item * TS + p];
    for (int j = 0; j < 8; ++j) {
      float z = 0.f;
      if (j < FD) {
        const float y = ys[((int64_t)item * TS + p) * FD + j];
        z = logf(y) - log1pf(-y);
      }
      S.zsnap[FK][p][j] = z;
    }
  }
  __syncthreads();
  // ---- inverse pass: z_K -> z_0, keeping the raw outputs of every layer
  for (int k = FK - 1; k >= 0; --k) {
    flow_load_layer(S.L, W, Bw, k, S.c);
    __syncthreads();
    // the forward MLP's raw outputs for the warp's 16 samples
    flow_mlp_st(S.L, k, &S.zsnap[k + 1][0][0], r0, &S.so[k][r0]);
    __syncthreads();
    for (int p = threadIdx.x; p < TS; p += blockDim.x) {
      const int nb = flow_nb(k);
      for (int j = 0; j < 8; ++j) S.zsnap[k][p][j] = S.zsnap[k + 1][p][j];
      for (int j = 0; j < nb; ++j) {
        const float s = F_SMAX * tanhf(S.so[k][p][j] * (1.f / F_SMAX));
        const int idx = flow_b(k, j);
        S.zsnap[k][p][idx] = (S.zsnap[k + 1][p][idx] - S.so[k][p][nb + j]) * __expf(-s);
      }
    }
    __syncthreads();
  }
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
        const float z0 = S.zsnap[0][p][j];
        lp += log_sig_prime(S.zsnap[FK][p][j]) - log_sig_prime(z0);  // full log|dy/du|
        const float sg = 1.f / (1.f + __expf(-z0));
        gzz = -S.w[p] * (1.f - 2.f * sg);
      }
      S.gz[p][j] = gzz;
    }
    lsum += S.w[p] * lp;
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) atomicAdd(loss_out, lsum);
  __syncthreads();
  // ---- backward, layer 0 upwards
  for (int k = 0; k < FK; ++k) {
    const int na = flow_na(k), nb = flow_nb(k);
    flow_load_layer(S.L, W, Bw, k, S.c);
    for (int n = threadIdx.x; n < FH; n += blockDim.x) S.colsum[n] = 0.f;
    __syncthreads();
    flow_train_recompute(S, k, S.zsnap[k + 1], r0);
    // per-sample output gradient g_o = (dL/ds_raw | dL/dt), and dL/dz_{k+1}[B]
    for (int p = threadIdx.x; p < TS; p += blockDim.x) {
      for (int j = 0; j < 8; ++j) S.GOt[j][p] = __float2bfloat16_rn(0.f);
      for (int j = 0; j < nb; ++j) {
        const int idx = flow_b(k, j);
        const float th = tanhf(S.so[k][p][j] * (1.f / F_SMAX));
        const float s = F_SMAX * th;
        const float tt = S.so[k][p][nb + j];
        const float e = __expf(-s);
        const float gzb = S.gz[p][idx];
        const float g_t = -gzb * e;
        const float g_s = -gzb * (S.zsnap[k + 1][p][idx] - tt) * e + S.w[p];
        S.GOt[j][p] = __float2bfloat16_rn(g_s * (1.f - th * th));
        S.GOt[nb + j][p] = __float2bfloat16_rn(g_t);
        S.gz[p][idx] = gzb * e;            // dL/dz_{k+1}[B]; [A] keeps the pass-through
      }
    }
    __syncthreads();
    // dW3 = h2^T g_o (M = 128 hidden, N = 8, K = 128 samples); db3 = sum g_o
    {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int m0 = warp * 16;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        uint32_t af[4];
        const int kr = kk * 16 + 2 * t;
        af[0] = ld_pair_T(&S.H2[0][0], FLD, kr, m0 + g);
        af[1] = ld_pair_T(&S.H2[0][0], FLD, kr, m0 + g + 8);
        af[2] = ld_pair_T(&S.H2[0][0], FLD, kr + 8, m0 + g);
        af[3] = ld_pair_T(&S.H2[0][0], FLD, kr + 8, m0 + g + 8);
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&S.GOt[g][kr]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&S.GOt[g][kr + 8]);
        mma_bf16(acc, af, b0, b1);
      }
      atomicAdd(&G->W3[k][m0 + g][2 * t], acc[0]);
      atomicAdd(&G->W3[k][m0 + g][2 * t + 1], acc[1]);
      atomicAdd(&G->W3[k][m0 + g + 8][2 * t], acc[2]);
      atomicAdd(&G->W3[k][m0 + g + 8][2 * t + 1], acc[3]);
      if (threadIdx.x < 8) {
        float s = 0.f;
        for (int p = 0; p < TS; ++p) s += __bfloat162float(S.GOt[threadIdx.x][p]);
        atomicAdd(&G->b3[k][threadIdx.x], s);
      }
    }
    // g_a2 = (g_o W3^T) * [a2 > 0] in FP32 (K = 8), stored BF16; db2 partials
    for (int e = threadIdx.x; e < TS * FH; e += blockDim.x) {
      const int p = e / FH, n = e % FH;
      float v = 0.f;
      if (__bfloat162float(S.H2[p][n]) > 0.f) {
#pragma unroll
        for (int o = 0; o < 8; ++o) v = fmaf(__bfloat162float(S.GOt[o][p]), __bfloat162float(S.L.W3t[o][n]), v);
      }
      S.GA2[p][n] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    for (int n = threadIdx.x; n < FH; n += blockDim.x) {
      float s = 0.f;
      for (int p = 0; p < TS; ++p) s += __bfloat162float(S.GA2[p][n]);
      atomicAdd(&G->b2[k][n], s);
    }
    // dW2 = h1^T g_a2 (M = 128 in, N = 128 out, K = 128 samples)
    {
      const int m0 = warp * 16;
      uint32_t af[8][4];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int kr = kk * 16 + 2 * t;
        af[kk][0] = ld_pair_T(&S.H1[0][0], FLD, kr, m0 + g);
        af[kk][1] = ld_pair_T(&S.H1[0][0], FLD, kr, m0 + g + 8);
        af[kk][2] = ld_pair_T(&S.H1[0][0], FLD, kr + 8, m0 + g);
        af[kk][3] = ld_pair_T(&S.H1[0][0], FLD, kr + 8, m0 + g + 8);
      }
#pragma unroll 1
      for (int j = 0; j < 16; ++j) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int kr = kk * 16 + 2 * t;
          const uint32_t b0 = ld_pair_T(&S.GA2[0][0], FLD, kr, j * 8 + g);
          const uint32_t b1 = ld_pair_T(&S.GA2[0][0], FLD, kr + 8, j * 8 + g);
          mma_bf16(acc, af[kk], b0, b1);
        }
        const int c0 = j * 8 + 2 * t;
        atomicAdd(&G->W2[k][m0 + g][c0], acc[0]);
        atomicAdd(&G->W2[k][m0 + g][c0 + 1], acc[1]);
        atomicAdd(&G->W2[k][m0 + g + 8][c0], acc[2]);
        atomicAdd(&G->W2[k][m0 + g + 8][c0 + 1], acc[3]);
      }
    }
    // g_h1 = g_a2 W2^T (M = 128 samples, N = 128 in, K = 128 out), then g_a1 = g_h1 [a1 > 0]
    {
      uint32_t af[8][4];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int c0 = kk * 16 + 2 * t;
        af[kk][0] = *reinterpret_cast<const uint32_t*>(&S.GA2[r0 + g][c0]);
        af[kk][1] = *reinterpret_cast<const uint32_t*>(&S.GA2[r0 + g + 8][c0]);
        af[kk][2] = *reinterpret_cast<const uint32_t*>(&S.GA2[r0 + g][c0 + 8]);
        af[kk][3] = *reinterpret_cast<const uint32_t*>(&S.GA2[r0 + g + 8][c0 + 8]);
      }
      float za0[4], za1[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        za0[j] = j < na ? S.zsnap[k + 1][r0 + g][flow_a(k, j)] : 0.f;
        za1[j] = j < na ? S.zsnap[k + 1][r0 + g + 8][flow_a(k, j)] : 0.f;
      }
      float gzA0[4] = {0.f, 0.f, 0.f, 0.f}, gzA1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
      for (int j = 0; j < 16; ++j) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int kr = kk * 16 + 2 * t;
          // B[k = out][n = in] = W2[in][out] = W2t[out][in]
          const uint32_t b0 = ld_pair_T(&S.L.W2t[0][0], FLD, kr, j * 8 + g);
          const uint32_t b1 = ld_pair_T(&S.L.W2t[0][0], FLD, kr + 8, j * 8 + g);
          mma_bf16(acc, af[kk], b0, b1);
        }
        // rows r0+g (acc 0,1) and r0+g+8 (acc 2,3); columns c0, c0+1
        const int c0 = j * 8 + 2 * t;
        float ga[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int col = c0 + (q & 1);
          const float* zz = (q < 2) ? za0 : za1;
          float a1 = S.L.cb1[col];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) a1 = fmaf(zz[jj], S.L.W1a[jj][col], a1);
          ga[q] = a1 > 0.f ? acc[q] : 0.f;
        }
        // dW1a[a][col] += za[a] g_a1 over the two rows; dz_A += g_a1 W1a^T
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = c0 + q;
          float colv = ga[q] + ga[q + 2];
          for (int o = 4; o < 32; o <<= 1) colv += __shfl_xor_sync(0xffffffffu, colv, o);
          if (g == 0) atomicAdd(&S.colsum[col], colv);
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            float dv = za0[jj] * ga[q] + za1[jj] * ga[q + 2];
            for (int o = 4; o < 32; o <<= 1) dv += __shfl_xor_sync(0xffffffffu, dv, o);
            if (g == 0 && jj < na) atomicAdd(&G->W1a[k][jj][col], dv);
            gzA0[jj] = fmaf(ga[q], S.L.W1a[jj][col], gzA0[jj]);
            gzA1[jj] = fmaf(ga[q + 2], S.L.W1a[jj][col], gzA1[jj]);
          }
        }
      }
      // reduce dz_A over the 4 threads of a row (t) and add to the pass-through term
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        for (int o = 1; o < 4; o <<= 1) {
          gzA0[jj] += __shfl_xor_sync(0xffffffffu, gzA0[jj], o);
          gzA1[jj] += __shfl_xor_sync(0xffffffffu, gzA1[jj], o);
        }
      }
      if (t == 0) {
        for (int jj = 0; jj < na; ++jj) {
          S.gz[r0 + g][flow_a(k, jj)] += gzA0[jj];
          S.gz[r0 + g + 8][flow_a(k, jj)] += gzA1[jj];
        }
      }
    }
    __syncthreads();
    // b1 and W1c (the conditioning vector is constant over the CTA)
    for (int n = threadIdx.x; n < FH; n += blockDim.x) {
      const float cs_n = S.colsum[n];
      atomicAdd(&G->b1[k][n], cs_n);
      for (int q = 0; q < FC; ++q) atomicAdd(&G->W1c[k][q][n], S.c[q] * cs_n);
    }
    __syncthreads();
  }
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
