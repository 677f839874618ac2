// Learned importance sampler: parameter handle, BF16 operand refresh, forward
// map entry point (exact log-Jacobian), training kernels and Adam.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include "../../include/mem.h"
#include "mem_flow.cuh"
#include "mem_flow_train.cuh"
#include "mem_internal.h"

namespace mem {

__global__ void k_flow_bf16(const FlowW* __restrict__ W, FlowB* __restrict__ B) {
  const int k = blockIdx.x;
  for (int t = threadIdx.x; t < FH * FLD; t += blockDim.x) {
    const int o = t / FLD, i = t % FLD;
    B->W2t[k][o][i] = __float2bfloat16_rn(i < FH ? W->W2[k][i][o] : 0.f);
  }
  for (int t = threadIdx.x; t < 8 * FLD; t += blockDim.x) {
    const int o = t / FLD, i = t % FLD;
    B->W3t[k][o][i] = __float2bfloat16_rn(i < FH ? W->W3[k][i][o] : 0.f);
  }
  // first layer, K = 16: [W1a_hi | W1a_hi | W1a_lo | 0] (W1a rows past |A| are zero)
  for (int t = threadIdx.x; t < FH * FW1; t += blockDim.x) {
    const int o = t / FW1, i = t % FW1, q = i >> 2;
    const float v = i < 12 ? W->W1a[k][i & 3][o] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    B->W1t[k][o][i] = q <= 1 ? hi : (q == 2 ? lo : __float2bfloat16_rn(0.f));
    if (i < 16) B->W1u[k][umma_kmajor(o, i, 16)] = B->W1t[k][o][i];
  }
  // the output layer as the tcgen05 operand (N 16: outputs 8-15 zero)
  for (int t = threadIdx.x; t < 16 * FH; t += blockDim.x) {
    const int n = t / FH, i = t % FH;
    B->W3u[k][umma_kmajor(n, i, FH)] = __float2bfloat16_rn(n < 8 ? W->W3[k][i][n] : 0.f);
  }
  // the hidden layer as the tcgen05 operand, bias folded into k 128 (high) and 129 (low)
  for (int t = threadIdx.x; t < FH * FKH; t += blockDim.x) {
    const int n = t / FKH, i = t % FKH;
    __nv_bfloat16 v;
    if (i < FH) {
      v = __float2bfloat16_rn(W->W2[k][i][n]);
    } else {
      const float b = W->b2[k][n];
      const __nv_bfloat16 hi = __float2bfloat16_rn(b);
      v = i == FH ? hi : (i == FH + 1 ? __float2bfloat16_rn(b - __bfloat162float(hi))
                                      : __float2bfloat16_rn(0.f));
    }
    B->W2u[k][umma_kmajor(n, i, FKH)] = v;
  }
  // W2 with rows = inputs, K = outputs (the training's backward product)
  for (int t = threadIdx.x; t < FH * FH; t += blockDim.x) {
    const int n = t / FH, i = t % FH;
    B->W2v[k][umma_kmajor(n, i, FH)] = __float2bfloat16_rn(W->W2[k][n][i]);
  }
}

cudaError_t set_train_wait_limit(uint32_t polls) {
  return cudaMemcpyToSymbol(c_train_wait_limit, &polls, sizeof(polls));
}

// Forward map of n points sharing one conditioning vector: 128 points per CTA.
__global__ void __launch_bounds__(128) k_flow_map(const FlowW* __restrict__ W,
                                                   const FlowB* __restrict__ Bw, const float* cond,
                                                   const float* __restrict__ u, int64_t n,
                                                   float* __restrict__ y, float* __restrict__ logj) {
  __shared__ FlowInferLayer L;
  __shared__ float zs[64 * 8];
  __shared__ float c[FC];
  const int64_t base = (int64_t)blockIdx.x * 64;
  if (threadIdx.x < FC) c[threadIdx.x] = cond[threadIdx.x];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) {
    const int64_t i = base + t;
    float lj = 0.f;
    for (int j = 0; j < FD; ++j) {
      const float uu = i < n ? u[i * FD + j] : 0.5f;
      const float z = logf(uu) - log1pf(-uu);
      zs[t * 8 + j] = z;
      lj -= log_sig_prime(z);
    }
    zs[t * 8 + 7] = lj;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  for (int k = 0; k < FK; ++k) {
    flow_load_infer(L, W, Bw, k, c);
    __syncthreads();
    flow_layer_rows<1>(L, k, zs, warp * 16);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < 64; t += blockDim.x) {
    const int64_t i = base + t;
    if (i >= n) continue;
    float lj = zs[t * 8 + 7];
    for (int j = 0; j < FD; ++j) {
      const float z = zs[t * 8 + j];
      y[i * FD + j] = 1.f / (1.f + __expf(-z));
      lj += log_sig_prime(z);
    }
    logj[i] = lj;
  }
}

}  // namespace mem

using namespace mem;

namespace {

mem_status ffail(mem_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

// natural flat layout <-> padded FlowW
void flat_to_padded(const float* p, FlowW& W) {
  std::memset(&W, 0, sizeof(W));
  for (int k = 0; k < FK; ++k) {
    const int na = flow_na(k), nb = flow_nb(k);
    for (int a = 0; a < na; ++a)
      for (int h = 0; h < FH; ++h) W.W1a[k][a][h] = *p++;
    for (int q = 0; q < FC; ++q)
      for (int h = 0; h < FH; ++h) W.W1c[k][q][h] = *p++;
    for (int h = 0; h < FH; ++h) W.b1[k][h] = *p++;
    for (int i = 0; i < FH; ++i)
      for (int o = 0; o < FH; ++o) W.W2[k][i][o] = *p++;
    for (int h = 0; h < FH; ++h) W.b2[k][h] = *p++;
    for (int i = 0; i < FH; ++i)
      for (int o = 0; o < 2 * nb; ++o) W.W3[k][i][o] = *p++;
    for (int o = 0; o < 2 * nb; ++o) W.b3[k][o] = *p++;
  }
}

void padded_to_flat(const FlowW& W, float* p) {
  for (int k = 0; k < FK; ++k) {
    const int na = flow_na(k), nb = flow_nb(k);
    for (int a = 0; a < na; ++a)
      for (int h = 0; h < FH; ++h) *p++ = W.W1a[k][a][h];
    for (int q = 0; q < FC; ++q)
      for (int h = 0; h < FH; ++h) *p++ = W.W1c[k][q][h];
    for (int h = 0; h < FH; ++h) *p++ = W.b1[k][h];
    for (int i = 0; i < FH; ++i)
      for (int o = 0; o < FH; ++o) *p++ = W.W2[k][i][o];
    for (int h = 0; h < FH; ++h) *p++ = W.b2[k][h];
    for (int i = 0; i < FH; ++i)
      for (int o = 0; o < 2 * nb; ++o) *p++ = W.W3[k][i][o];
    for (int o = 0; o < 2 * nb; ++o) *p++ = W.b3[k][o];
  }
}

}  // namespace

extern "C" {

int64_t mem_flow_param_count(void) {
  int64_t n = 0;
  for (int k = 0; k < FK; ++k) n += flow_layer_params(k);
  return n;
}

mem_status mem_flow_create(uint64_t seed, mem_flow** out) {
  if (!out) return ffail(MEM_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  // He-style initialisation; output layer zero so the flow starts as the identity map
  std::vector<float> flat(mem_flow_param_count());
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  float* p = flat.data();
  for (int k = 0; k < FK; ++k) {
    const int na = flow_na(k), nb = flow_nb(k);
    const float s1 = 1.f / std::sqrt((float)(na + FC)), s2 = 1.f / std::sqrt((float)FH);
    for (int i = 0; i < (na + FC) * FH; ++i) *p++ = s1 * nd(rng);
    for (int i = 0; i < FH; ++i) *p++ = 0.f;
    for (int i = 0; i < FH * FH; ++i) *p++ = s2 * nd(rng);
    for (int i = 0; i < FH; ++i) *p++ = 0.f;
    for (int i = 0; i < FH * 2 * nb + 2 * nb; ++i) *p++ = 0.f;
  }
  mem_flow* f = new mem_flow;
  f->magic = MAGIC_FLOW;
  cudaGetDevice(&f->device);
  f->W = nullptr;
  f->B = nullptr;
  f->m = f->v = nullptr;
  f->grad = nullptr;
  f->step = 0;
  cudaError_t e = cudaMalloc(&f->W, sizeof(FlowW));
  if (e == cudaSuccess) e = cudaMalloc(&f->B, sizeof(FlowB));
  if (e == cudaSuccess) e = cudaMalloc(&f->m, sizeof(FlowW));
  if (e == cudaSuccess) e = cudaMalloc(&f->v, sizeof(FlowW));
  if (e == cudaSuccess) e = cudaMalloc(&f->grad, sizeof(FlowW));
  if (e == cudaSuccess) e = cudaMemset(f->m, 0, sizeof(FlowW));
  if (e == cudaSuccess) e = cudaMemset(f->v, 0, sizeof(FlowW));
  if (e != cudaSuccess) {
    cudaFree(f->W); cudaFree(f->B); cudaFree(f->m); cudaFree(f->v); cudaFree(f->grad);
    delete f;
    return ffail(MEM_ERR_OOM, "flow allocation");
  }
  *out = f;
  return mem_flow_set_params(f, flat.data(), (int64_t)flat.size());
}

mem_status mem_flow_set_params(mem_flow* f, const float* params, int64_t n) {
  if (!f || f->magic != MAGIC_FLOW || !params || n != mem_flow_param_count())
    return ffail(MEM_ERR_INVALID_ARG, "invalid flow handle or parameter count");
  std::vector<FlowW> h(1);
  flat_to_padded(params, h[0]);
  cudaError_t e = cudaMemcpy(f->W, h.data(), sizeof(FlowW), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_flow_bf16<<<FK, 256>>>(f->W, f->B);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return ffail(MEM_ERR_CUDA, std::string("mem_flow_set_params: ") + cudaGetErrorString(e));
  return MEM_OK;
}

mem_status mem_flow_get_params(const mem_flow* f, float* params, int64_t n) {
  if (!f || f->magic != MAGIC_FLOW || !params || n != mem_flow_param_count())
    return ffail(MEM_ERR_INVALID_ARG, "invalid flow handle or parameter count");
  std::vector<FlowW> h(1);
  cudaError_t e = cudaMemcpy(h.data(), f->W, sizeof(FlowW), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ffail(MEM_ERR_CUDA, "mem_flow_get_params");
  padded_to_flat(h[0], params);
  return MEM_OK;
}

mem_status mem_flow_map(const mem_flow* f, const float* cond, const float* u, int64_t n, float* y,
                        float* logj, void* stream) {
  if (!f || f->magic != MAGIC_FLOW || !cond || !u || !y || !logj || n < 1)
    return ffail(MEM_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((n + 63) / 64);
  k_flow_map<<<blocks, 128, 0, st>>>(f->W, f->B, cond, u, n, y, logj);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ffail(MEM_ERR_CUDA, std::string("mem_flow_map: ") + cudaGetErrorString(e));
  return MEM_OK;
}

namespace {

static_assert(sizeof(FlowTrainSmem) <= 227 * 1024, "training CTA shared memory above 227 KB");

// set on every call: the attribute belongs to the current device's context
cudaError_t train_smem_attr() {
  return cudaFuncSetAttribute(k_flow_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(FlowTrainSmem));
}

// per-CTA z snapshots of the training kernel (FK + 1 levels x TS samples x 8)
constexpr size_t ZSCR_PER_CTA = (size_t)(FK + 1) * TS * 8;

}  // namespace

mem_status mem_flow_grad(mem_flow* f, const float* ys, const float* ws, const float* cs,
                         int64_t n_items, float* grad, double* loss, void* stream) {
  if (!f || f->magic != MAGIC_FLOW || !ys || !ws || !cs || !grad || n_items < 1)
    return ffail(MEM_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> b(n_items);
  for (int64_t i = 0; i < n_items; ++i) b[i] = (int32_t)i;
  int32_t* db = nullptr;
  float* dl = nullptr;
  float* zscr = nullptr;
  int* derr = nullptr;
  int herr = 0;
  cudaError_t e = train_smem_attr();
  if (e == cudaSuccess) e = cudaMalloc(&db, n_items * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&zscr, (size_t)n_items * ZSCR_PER_CTA * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(db, b.data(), n_items * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dl, 0, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(f->grad, 0, sizeof(FlowW), st);
  if (e == cudaSuccess) {
    k_flow_train<<<(unsigned)n_items, 256, sizeof(FlowTrainSmem), st>>>(
        f->W, f->B, ys, ws, cs, db, reinterpret_cast<FlowW*>(f->grad), dl, zscr, derr);
    e = cudaGetLastError();
  }
  std::vector<FlowW> h(1);
  float lh = 0.f;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), f->grad, sizeof(FlowW), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&lh, dl, sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(db);
  cudaFree(dl);
  cudaFree(zscr);
  cudaFree(derr);
  if (e != cudaSuccess) return ffail(MEM_ERR_CUDA, std::string("mem_flow_grad: ") + cudaGetErrorString(e));
  if (herr) return ffail(MEM_ERR_TIMEOUT, "mem_flow_grad: a tensor-core wait gave up");
  padded_to_flat(h[0], grad);
  if (loss) *loss = lh;
  return MEM_OK;
}

mem_status mem_flow_train(mem_flow* f, const float* ys, const float* ws, const float* cs,
                          int64_t n_items, int32_t n_steps, int32_t batch_items, float lr,
                          uint64_t seed, float* loss_trace, void* stream) {
  if (!f || f->magic != MAGIC_FLOW || !ys || !ws || !cs || n_items < 1 || n_steps < 1 ||
      batch_items < 1 || batch_items > n_items || !(lr > 0.f))
    return ffail(MEM_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  // batches: a fresh random permutation of the items per epoch (host RNG, uploaded once)
  std::mt19937_64 rng(seed);
  std::vector<int32_t> order(n_items), batches((size_t)n_steps * batch_items);
  int64_t pos = n_items;
  for (int s = 0; s < n_steps; ++s)
    for (int b = 0; b < batch_items; ++b) {
      if (pos >= n_items) {
        for (int64_t i = 0; i < n_items; ++i) order[i] = (int32_t)i;
        std::shuffle(order.begin(), order.end(), rng);
        pos = 0;
      }
      batches[(size_t)s * batch_items + b] = order[pos++];
    }
  int32_t* db = nullptr;
  float* dl = nullptr;
  float* zscr = nullptr;
  int* derr = nullptr;
  int herr = 0;
  cudaError_t e = train_smem_attr();
  if (e == cudaSuccess) e = cudaMalloc(&db, batches.size() * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&dl, (size_t)n_steps * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&zscr, (size_t)batch_items * ZSCR_PER_CTA * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(db, batches.data(), batches.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dl, 0, (size_t)n_steps * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->grad, 0, sizeof(FlowW), st);
  const int64_t nparam = (int64_t)(sizeof(FlowW) / sizeof(float));
  const float b1 = 0.9f, b2 = 0.999f;
  for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
    k_flow_train<<<batch_items, 256, sizeof(FlowTrainSmem), st>>>(
        f->W, f->B, ys, ws, cs, db + (size_t)s * batch_items, reinterpret_cast<FlowW*>(f->grad),
        dl + s, zscr, derr);
    ++f->step;
    const float bc1 = 1.f - std::pow(b1, (float)f->step), bc2 = 1.f - std::pow(b2, (float)f->step);
    k_flow_adam<<<256, 256, 0, st>>>(f->W, f->m, f->v, reinterpret_cast<FlowW*>(f->grad), nparam,
                                     lr, b1, b2, 1e-8f, bc1, bc2, 1.f / batch_items);
    k_flow_bf16<<<FK, 256, 0, st>>>(f->W, f->B);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && loss_trace)
    e = cudaMemcpy(loss_trace, dl, (size_t)n_steps * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(db);
  cudaFree(dl);
  cudaFree(zscr);
  cudaFree(derr);
  if (e != cudaSuccess) return ffail(MEM_ERR_CUDA, std::string("mem_flow_train: ") + cudaGetErrorString(e));
  if (herr) return ffail(MEM_ERR_TIMEOUT, "mem_flow_train: a tensor-core wait gave up");
  return MEM_OK;
}

}  // extern "C"

void mem_flow_release(mem_flow* f) {
  cudaFree(f->W);
  cudaFree(f->B);
  cudaFree(f->m);
  cudaFree(f->v);
  cudaFree(f->grad);
  f->magic = 0;
  delete f;
}
