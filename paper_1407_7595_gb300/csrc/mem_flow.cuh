// Learned importance sampler: an event-conditioned affine-coupling flow on the
// unit cube that replaces the VEGAS map of the Monte Carlo integral (Sec. 2,
// importance sampling) for the ttbar integrand.
//
//   u ~ U(0,1)^7 -> z = logit(u) -> 6 coupling layers -> y = sigmoid(z) -> physics map
//   layer k: z[B] <- z[B] exp(s) + t, (s_raw, t) = MLP_k(z[A], c), s = 2 tanh(s_raw / 2)
//   MLP: Linear(|A| + 16 -> 128), ReLU, Linear(128 -> 128), ReLU, Linear(128 -> 2|B|)
//   A = coordinates with parity k % 2, B = the rest; c = 16 measured-momentum features
//   log|dy/du| = sum log sigmoid'(z_out) + sum_k sum_B s - sum log sigmoid'(z_in)  (exact)
//
// Tensor cores: the sampling kernels (mem_flow_int.cuh) and the training kernel
// (mem_flow_train.cuh) run the first and hidden products on tcgen05 with tensor-
// memory accumulators; the sampling kernels' 8-wide output layer stays on warp-
// level mma.sync, where a tensor-memory round trip costs more than the product.
// The small forward map entry point (mem_flow_map) runs every layer as mma.sync
// m16n8k16 on 16-point row blocks (flow_layer_rows below). The training kernel
// evaluates the first layer (K = |A| <= 4) in FP32; inference runs it as a
// K = 16 product of a two-part BF16 split of z_A and of W1a (~16 bits kept).
#pragma once
#include "mem_fastmath.cuh"
#include <cuda_bf16.h>

#include "mem_common.cuh"

namespace mem {

constexpr int FK = 6;            // coupling layers
constexpr int FH = 128;          // hidden width
constexpr int FC = 16;           // conditioning features
constexpr int FD = 7;            // dimensions (ttbar)
constexpr int FLD = FH + 8;      // padded BF16 row stride (conflict-free fragment loads)
constexpr int FW1 = 24;          // padded row of the first-layer BF16 operand (16 used)
constexpr int FKH = FH + 16;     // K of the tcgen05 hidden product: 128 inputs, 1, 1, 14 zeros
constexpr float F_SMAX = 2.f;

__host__ __device__ constexpr int flow_na(int k) { return k % 2 == 0 ? (FD + 1) / 2 : FD / 2; }
__host__ __device__ constexpr int flow_nb(int k) { return FD - flow_na(k); }
// j-th coordinate of the A (resp. B) set of layer k
__host__ __device__ constexpr int flow_a(int k, int j) { return 2 * j + (k & 1); }
__host__ __device__ constexpr int flow_b(int k, int j) { return 2 * j + 1 - (k & 1); }

// FP32 master parameters (padded layouts: |A| -> 4 rows, 2|B| -> 8 outputs).
struct FlowW {
  float W1a[FK][4][FH];
  float W1c[FK][FC][FH];
  float b1[FK][FH];
  float W2[FK][FH][FH];   // [in][out]
  float b2[FK][FH];
  float W3[FK][FH][8];    // [in][out]
  float b3[FK][8];
};
// BF16 operand copies, [out][in] with padded rows. W1t is the first layer as a
// K = 16 operand for z_A split into two BF16 parts (z = z_hi + z_lo):
// k 0-3 = W1a_hi (times z_hi), 4-7 = W1a_hi (times z_lo), 8-11 = W1a_lo
// (times z_hi), 12-15 = 0, so the product keeps ~16 significant bits.
// W2u is the hidden layer as a tcgen05 B operand (N 128 x K 144, K-major, no
// swizzle; see umma_kmajor) with its bias folded in: k 0-127 = W2[k][n],
// k 128 = b2 high part, k 129 = b2 low part (BF16 split, ~16 bits), k 130-143
// = 0; the activation operand carries 1, 1, 0 ... in those columns.
// W1u and W3u are the first and output layers as tcgen05 B operands (same
// layout): W1u N 128 x K 16 in the split form of W1t; W3u N 16 x K 128, rows
// n < 8 = W3[k][.][n], rows 8-15 zero; W2v below.
struct FlowB {
  __nv_bfloat16 W2t[FK][FH][FLD];
  __nv_bfloat16 W3t[FK][8][FLD];
  __nv_bfloat16 W1t[FK][FH][FW1];
  __nv_bfloat16 W2u[FK][FH * FKH];
  __nv_bfloat16 W1u[FK][FH * 16];
  __nv_bfloat16 W3u[FK][16 * FH];
  __nv_bfloat16 W2v[FK][FH * FH];   // W2 as the B operand of dL/dh1 = dL/da2 W2^T (training):
                                    // N 128 (in) x K 128 (out), K-major, no swizzle
};

// Element index of (row m, column k) of a K-column tile in the tcgen05
// canonical K-major layout without swizzle: core matrices of 8 rows x 8
// elements (128 bytes); LBO = 128 bytes along K, SBO = 16 K bytes along rows.
__host__ __device__ constexpr int umma_kmajor(int m, int k, int K) {
  return (m >> 3) * (8 * K) + (k >> 3) * 64 + (m & 7) * 8 + (k & 7);
}
// Natural (unpadded) FP32 parameter count, the order of the flat host layout.
__host__ __device__ constexpr int flow_layer_params(int k) {
  return flow_na(k) * FH + FC * FH + FH + FH * FH + FH + FH * 2 * flow_nb(k) + 2 * flow_nb(k);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Two floats -> ReLU -> BF16 pair (lo in the low half), one conversion.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float log_sig_prime(float z) {
  // log(sigmoid(z)(1 - sigmoid(z))) = -|z| - 2 log(1 + e^-|z|)
  const float a = fabsf(z);
  return -a - 2.f * log1pf(__expf(-a));
}

// ---------------------------------------------------------------------------
// Inference form: all three layers on the tensor cores, RB 16-row blocks per
// warp sharing each weight fragment, s and t exchanged by warp shuffles.
// ---------------------------------------------------------------------------
struct __align__(16) FlowInferLayer {
  __nv_bfloat16 W2t[FH][FLD];
  __nv_bfloat16 W3t[8][FLD];
  __nv_bfloat16 W1t[FH][FW1];
  float cb1[FH];   // c W1c + b1 for the CTA's item
  float b2[FH];
  float b3[8];
};

__device__ inline void flow_load_infer(FlowInferLayer& L, const FlowW* __restrict__ W,
                                       const FlowB* __restrict__ Bw, int k, const float* c) {
  const uint4* src = reinterpret_cast<const uint4*>(&Bw->W2t[k][0][0]);
  uint4* dst = reinterpret_cast<uint4*>(&L.W2t[0][0]);
  for (int t = threadIdx.x; t < (int)(sizeof(L.W2t) / 16); t += blockDim.x) dst[t] = src[t];
  const uint4* src3 = reinterpret_cast<const uint4*>(&Bw->W3t[k][0][0]);
  uint4* dst3 = reinterpret_cast<uint4*>(&L.W3t[0][0]);
  for (int t = threadIdx.x; t < (int)(sizeof(L.W3t) / 16); t += blockDim.x) dst3[t] = src3[t];
  const uint4* src1 = reinterpret_cast<const uint4*>(&Bw->W1t[k][0][0]);
  uint4* dst1 = reinterpret_cast<uint4*>(&L.W1t[0][0]);
  for (int t = threadIdx.x; t < (int)(sizeof(L.W1t) / 16); t += blockDim.x) dst1[t] = src1[t];
  for (int n = threadIdx.x; n < FH; n += blockDim.x) {
    float s = W->b1[k][n];
#pragma unroll
    for (int q = 0; q < FC; ++q) s = fmaf(c[q], W->W1c[k][q][n], s);
    L.cb1[n] = s;
    L.b2[n] = W->b2[k][n];
  }
  if (threadIdx.x < 8) L.b3[threadIdx.x] = W->b3[k][threadIdx.x];
}

__device__ __forceinline__ float bf16_hi(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// z_B <- z_B e^s + t for one row from the 8 raw outputs (compile-time |B|).
template <int NB>
__device__ __forceinline__ void flow_update_row(float* zr, const float (&v)[8], int k) {
  float ls = 0.f;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const float s = F_SMAX * tanh_coupling(v[j] * (1.f / F_SMAX));
    const int idx = flow_b(k, j);
    zr[idx] = fmaf(zr[idx], __expf(s), v[NB + j]);
    ls += s;
  }
  zr[7] += ls;
}

// One warp: coupling layer k on the RB x 16 rows r0 .. of zs (row stride 8):
// MLP on the tensor cores, then the affine update and the log-Jacobian.
template <int RB>
__device__ inline void flow_layer_rows(const FlowInferLayer& L, int k, float* zs, int r0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int na = flow_na(k);
  // first layer: A = [z_A hi | z_A lo | z_A hi | 0] (K = 16); lane t holds
  // columns 2t, 2t+1 (a0, a1) and 2t+8, 2t+9 (a2, a3)
  const int j0 = (2 * t) & 3;
  uint32_t a[RB][8][4];
#pragma unroll
  for (int rb = 0; rb < RB; ++rb) {
    uint32_t a1[4];
    float zv[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = r0 + rb * 16 + g + 8 * h;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int j = j0 + q;
        zv[h][q] = j < na ? zs[row * 8 + flow_a(k, j)] : 0.f;
      }
    }
    if (t < 2) {
      a1[0] = pack_bf16(zv[0][0], zv[0][1]);
      a1[1] = pack_bf16(zv[1][0], zv[1][1]);
      a1[2] = a1[0];
      a1[3] = a1[1];
    } else {
      a1[0] = pack_bf16(zv[0][0] - bf16_hi(zv[0][0]), zv[0][1] - bf16_hi(zv[0][1]));
      a1[1] = pack_bf16(zv[1][0] - bf16_hi(zv[1][0]), zv[1][1] - bf16_hi(zv[1][1]));
      a1[2] = 0u;
      a1[3] = 0u;
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      float acc[2][4];
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int n0 = (2 * kk + h2) * 8;
        const float c0 = L.cb1[n0 + 2 * t], c1 = L.cb1[n0 + 2 * t + 1];
        acc[h2][0] = c0;
        acc[h2][1] = c1;
        acc[h2][2] = c0;
        acc[h2][3] = c1;
        const __nv_bfloat16* brow = &L.W1t[n0 + g][0];
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(brow + 2 * t);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(brow + 2 * t + 8);
        mma_bf16(acc[h2], a1, b0, b1);
      }
      a[rb][kk][0] = pack_bf16(fmaxf(acc[0][0], 0.f), fmaxf(acc[0][1], 0.f));
      a[rb][kk][1] = pack_bf16(fmaxf(acc[0][2], 0.f), fmaxf(acc[0][3], 0.f));
      a[rb][kk][2] = pack_bf16(fmaxf(acc[1][0], 0.f), fmaxf(acc[1][1], 0.f));
      a[rb][kk][3] = pack_bf16(fmaxf(acc[1][2], 0.f), fmaxf(acc[1][3], 0.f));
    }
  }
  // hidden layer (K = 128) and output layer, weight fragments shared by the row blocks
  float o[RB][4];
#pragma unroll
  for (int rb = 0; rb < RB; ++rb) o[rb][0] = o[rb][1] = o[rb][2] = o[rb][3] = 0.f;
#pragma unroll 1
  for (int jp = 0; jp < 8; ++jp) {
    float acc[RB][2][4];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int j = 2 * jp + h2;
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) acc[rb][h2][0] = acc[rb][h2][1] = acc[rb][h2][2] = acc[rb][h2][3] = 0.f;
      const __nv_bfloat16* brow = &L.W2t[j * 8 + g][0];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(brow + kk * 16 + 2 * t);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(brow + kk * 16 + 2 * t + 8);
#pragma unroll
        for (int rb = 0; rb < RB; ++rb) mma_bf16(acc[rb][h2], a[rb][kk], b0, b1);
      }
      const float bb0 = L.b2[j * 8 + 2 * t], bb1 = L.b2[j * 8 + 2 * t + 1];
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) {
        acc[rb][h2][0] = fmaxf(acc[rb][h2][0] + bb0, 0.f);
        acc[rb][h2][1] = fmaxf(acc[rb][h2][1] + bb1, 0.f);
        acc[rb][h2][2] = fmaxf(acc[rb][h2][2] + bb0, 0.f);
        acc[rb][h2][3] = fmaxf(acc[rb][h2][3] + bb1, 0.f);
      }
    }
    const __nv_bfloat16* brow3 = &L.W3t[g][0];
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(brow3 + jp * 16 + 2 * t);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(brow3 + jp * 16 + 2 * t + 8);
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
      uint32_t a2[4];
      a2[0] = pack_bf16(acc[rb][0][0], acc[rb][0][1]);
      a2[1] = pack_bf16(acc[rb][0][2], acc[rb][0][3]);
      a2[2] = pack_bf16(acc[rb][1][0], acc[rb][1][1]);
      a2[3] = pack_bf16(acc[rb][1][2], acc[rb][1][3]);
      mma_bf16(o[rb], a2, b0, b1);
    }
  }
  // raw outputs (s_raw | t) of rows g and g + 8 to lanes t = 0 and t = 1 of the quad
  const float bo0 = L.b3[2 * t], bo1 = L.b3[2 * t + 1];
#pragma unroll
  for (int rb = 0; rb < RB; ++rb) {
    const float v0 = o[rb][0] + bo0, v1 = o[rb][1] + bo1, v2 = o[rb][2] + bo0, v3 = o[rb][3] + bo1;
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
      float* zr = zs + (r0 + rb * 16 + g + 8 * t) * 8;
      if (k & 1) flow_update_row<FD / 2 + 1>(zr, v, k);
      else flow_update_row<FD / 2>(zr, v, k);
    }
  }
  __syncwarp();
}

}  // namespace mem
