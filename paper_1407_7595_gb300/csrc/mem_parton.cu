// Parton-level ttbar weights (Sec. 4, "parton level"): every final-state momentum
// of the event is known, so every transfer function is a delta function and the
// method reduces to one evaluation of the PDF-weighted |M|^2 density per
// assignment of the two b quarks, averaged over the assignments (the paper's
// Table "time_parton" times this step for 1e5 events).
//
// One thread per event computes both assignments: the six massless lab momenta
// from (E, eta, phi), the resonance virtualities from pairwise
// 1 - cos(theta) = |n_i - n_j|^2 / 2 (sums of positive terms: no cancellation
// near the poles), the transverse boost to zero total pT, x1 and x2, the
// helicity-summed g g and q qbar squared amplitudes shared with the integrand
// (tt_amp2, once per assignment), the parton densities and the flux; the boost,
// x1, x2 and the densities are shared by the assignments. FP32 throughout; the constant
// factors ((2 pi)^4 2/s, the six 1/(2 (2 pi)^3) and the (m G)^4 of the four
// normalised propagators) are applied in FP64.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/mem.h"
#include "mem_internal.h"
#include "mem_ttbar.cuh"

namespace mem {
namespace {

constexpr int PARTON_THREADS = 256;
// resident CTAs per SM the kernel is built for (<= 128 registers)
constexpr int PARTON_MINB = 2;

struct LabP {
  float E, nx, ny, nz, lp, lm;   // energy, unit direction, 1 + tanh(eta), 1 - tanh(eta)
};

__device__ __forceinline__ LabP lab_of(float4 o) {
  LabP p;
  p.E = o.x;
  float sp, cp;
  sincosf(o.z, &sp, &cp);
  const float eh = expf(o.y), e2 = eh * eh;
  const float inv = 1.f / (e2 + 1.f);
  const float sech = 2.f * eh * inv;
  p.nx = cp * sech;
  p.ny = sp * sech;
  p.nz = (e2 - 1.f) * inv;
  p.lp = 2.f * e2 * inv;
  p.lm = 2.f * inv;
  return p;
}

// 1 - n_a . n_b for unit vectors, as |n_a - n_b|^2 / 2
__device__ __forceinline__ float omc(const LabP& a, const LabP& b) {
  const float dx = a.nx - b.nx, dy = a.ny - b.ny, dz = a.nz - b.nz;
  return 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// (m G)^2 / |q^2 - m^2 + i m G|^2
__device__ __forceinline__ float prop_n(float q2, float m2, float mg) {
  const float d = q2 - m2;
  const float mg2 = mg * mg;
  return mg2 / fmaf(d, d, mg2);
}

__device__ __forceinline__ LCv boost_lab(const LabP& p, const TBoost& B) {
  return boost_lc(p.E, p.E * p.nx, p.E * p.ny, p.E * p.lp, p.E * p.lm, B);
}

// FP32 weights (without the FP64 constant) of one record for both b-quark
// assignments. The transverse boost, x1, x2, s-hat, the parton densities and the
// W propagators do not depend on the assignment and are computed once; 0 if a
// momentum fraction reaches 1.
__device__ void parton_weights2(const float4 (&o)[6], const ProcConst& P, float& w0, float& w1) {
  w0 = w1 = 0.f;
  const LabP l = lab_of(o[0]);
  const LabP j1 = lab_of(o[1]);
  const LabP j2 = lab_of(o[2]);
  const LabP d = lab_of(o[3]);
  const LabP u = lab_of(o[4]);
  const LabP n = lab_of(o[5]);
  // invariants from pairwise 1 - cos(theta): p_i.p_j = E_i E_j (1 - cos theta_ij)
  const float pln = l.E * n.E * omc(l, n), pdu = d.E * u.E * omc(d, u);
  const float p1l = j1.E * l.E * omc(j1, l), p1n = j1.E * n.E * omc(j1, n);
  const float p2l = j2.E * l.E * omc(j2, l), p2n = j2.E * n.E * omc(j2, n);
  const float p1d = j1.E * d.E * omc(j1, d), p1u = j1.E * u.E * omc(j1, u);
  const float p2d = j2.E * d.E * omc(j2, d), p2u = j2.E * u.E * omc(j2, u);
  const float props_w = prop_n(2.f * pln, P.mw2, P.mwgw) * prop_n(2.f * pdu, P.mw2, P.mwgw);
  // transverse boost of the final state to zero total pT
  const float Etot = j1.E + l.E + n.E + j2.E + d.E + u.E;
  const float Px = j1.E * j1.nx + l.E * l.nx + n.E * n.nx + j2.E * j2.nx + d.E * d.nx + u.E * u.nx;
  const float Py = j1.E * j1.ny + l.E * l.ny + n.E * n.ny + j2.E * j2.ny + d.E * d.ny + u.E * u.ny;
  const float Ppp = j1.E * j1.lp + l.E * l.lp + n.E * n.lp + j2.E * j2.lp + d.E * d.lp + u.E * u.lp;
  const float Ppm = j1.E * j1.lm + l.E * l.lm + n.E * n.lm + j2.E * j2.lm + d.E * d.lm + u.E * u.lm;
  const float pt2 = fmaf(Px, Px, Py * Py);
  const float shat_lab = fmaf(Ppp, Ppm, -pt2);
  const float Ep = sqrtf(fmaf(0.25f * (Ppp - Ppm), (Ppp - Ppm), shat_lab));
  TBoost B;
  B.gm1 = pt2 / (Ep * (Etot + Ep));
  B.gam = 1.f + B.gm1;
  B.g2 = B.gam * B.gam / (B.gam + 1.f);
  B.bx = Px / Etot;
  B.by = Py / Etot;
  const LCv cl = boost_lab(l, B), cn = boost_lab(n, B), cd = boost_lab(d, B);
  const LCv cu = boost_lab(u, B), c1 = boost_lab(j1, B), c2 = boost_lab(j2, B);
  const float k1p = ((c1.pp + c2.pp) + (cl.pp + cn.pp)) + (cd.pp + cu.pp);
  const float k2m = ((c1.pm + c2.pm) + (cl.pm + cn.pm)) + (cd.pm + cu.pm);
  const float x1 = k1p / P.sqrt_s, x2 = k2m / P.sqrt_s;
  if (!(x1 < 1.f && x2 < 1.f)) return;
  const float shat = k1p * k2m;
  PdfX f1, f2;
  pdf_pair(P, x1, x2, f1, f2);
  const float cgg = P.tt_gg * f1.g * f2.g;
  const float cqq = P.tt_qq * 2.f * fmaf(f1.q, f2.qb, f1.qb * f2.q);
  const float common = (4.f / shat) * props_w /
                       (((j1.E * l.E) * (n.E * j2.E)) * (d.E * u.E));
  const float m = sqrtf(P.mt2);
#pragma unroll 1
  for (int a = 0; a < 2; ++a) {
    const LCv& cb = a ? c2 : c1;
    const LCv& cbb = a ? c1 : c2;
    const float pbl = a ? p2l : p1l, pbn = a ? p2n : p1n;
    const float pbd = a ? p1d : p2d, pbu = a ? p1u : p2u;
    const float props = prop_n(2.f * (pbl + pbn + pln), P.mt2, P.mtgt) *
                        prop_n(2.f * (pbd + pbu + pdu), P.mt2, P.mtgt);
    LCv tp, tm;
    tp.pp = cb.pp + cl.pp + cn.pp;
    tp.pm = cb.pm + cl.pm + cn.pm;
    tp.pt = cb.pt + cl.pt + cn.pt;
    tm.pp = cbb.pp + cd.pp + cu.pp;
    tm.pm = cbb.pm + cd.pm + cu.pm;
    tm.pt = cbb.pt + cd.pt + cu.pt;
    const TTAmp2 amp = tt_amp2(cl, cd, tp, tm, m, P.mt2, k1p, k2m, shat);
    const float w = fmaf(cgg, amp.gg, cqq * amp.qq) * common * pbn * pbu * props;
    if (a) w1 = w;
    else w0 = w;
  }
}

__device__ __forceinline__ bool record_ok(const float4 (&o)[6]) {
  bool ok = (o[0].w == 4.f || o[0].w == 2.f) && o[5].w == 6.f;
  for (int k = 1; k <= 4; ++k) ok = ok && o[k].w == 5.f;
  for (int k = 0; k < 6; ++k) ok = ok && o[k].x > 0.f && fabsf(o[k].y) < 40.f;
  return ok;
}

// One thread per event (grid-stride); pref_half = the FP64 constant / 2.
__global__ void __launch_bounds__(PARTON_THREADS, PARTON_MINB)
    k_parton_tt(const float* __restrict__ recs, int64_t n, const __grid_constant__ ProcConst P,
                double pref, double* __restrict__ prob, double* __restrict__ w_assign,
                int32_t* __restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const float4* r4 = reinterpret_cast<const float4*>(recs + e * REC);
    float4 o[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = __ldg(r4 + k);
    const bool ok = record_ok(o);
    float w0 = 0.f, w1 = 0.f;
    if (ok) parton_weights2(o, P, w0, w1);
    prob[e] = (0.5 * pref) * ((double)w0 + (double)w1);
    if (w_assign) {
      w_assign[2 * e] = pref * (double)w0;
      w_assign[2 * e + 1] = pref * (double)w1;
    }
    if (status) status[e] = ok ? MEM_OK : MEM_ERR_INVALID_ARG;
  }
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

mem_status pfail(mem_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

}  // namespace
}  // namespace mem

extern "C" mem_status mem_parton_weights(const mem_events* events, const mem_process* process,
                                         double* prob, double* w_assign, int32_t* ev_status,
                                         void* stream) {
  using namespace mem;
  if (!events || events->magic != MAGIC_EVT || !process || process->magic != MAGIC_PROC || !prob)
    return pfail(MEM_ERR_INVALID_ARG, "NULL or invalid handle/output");
  if (process->desc.kind != PROC_TTBAR || events->kind != PROC_TTBAR)
    return pfail(MEM_ERR_INVALID_ARG, "parton-level weights are defined for the ttbar process");
  const int64_t n = events->n;
  const bool dev = dev_ptr(prob);
  if ((w_assign && dev_ptr(w_assign) != dev) || (ev_status && dev_ptr(ev_status) != dev))
    return pfail(MEM_ERR_INVALID_ARG, "outputs must all be host or all be device memory");
  if (dev && ((uintptr_t)prob % alignof(double) || (uintptr_t)w_assign % alignof(double) ||
              (uintptr_t)ev_status % alignof(int32_t)))
    return pfail(MEM_ERR_INVALID_ARG, "device outputs must be aligned to their element size");
  cudaStream_t st = (cudaStream_t)stream;
  const ProcConst& P = process->pc;
  // (2 pi)^4 (2/s) prod_6 1/(2 (2 pi)^3) / ((m G)_t^4 (m G)_W^4), with the same FP32
  // m G as the kernel's normalised propagators
  const double tp = 2.0 * PI_D, s = process->desc.sqrt_s * process->desc.sqrt_s;
  const double mgt = (double)P.mtgt, mgw = (double)P.mwgw;
  const double pref = std::pow(tp, 4.0) * (2.0 / s) * std::pow(1.0 / (2.0 * std::pow(tp, 3.0)), 6.0) /
                      (mgt * mgt * mgt * mgt) / (mgw * mgw * mgw * mgw);
  // resident CTAs of the current device, cached per device (writers store equal values)
  static std::atomic<int> occ_cache[64];
  int dev_id = 0;
  cudaGetDevice(&dev_id);
  int full_ctas = dev_id < 64 ? occ_cache[dev_id].load(std::memory_order_relaxed) : 0;
  if (full_ctas == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_parton_tt, PARTON_THREADS, 0);
    full_ctas = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    if (dev_id < 64) occ_cache[dev_id].store(full_ctas, std::memory_order_relaxed);
  }
  const int64_t need = (n + PARTON_THREADS - 1) / PARTON_THREADS;
  const int64_t full = full_ctas;
  const unsigned grid = (unsigned)(need < full ? need : full);
  double* d_prob = prob;
  double* d_w = w_assign;
  int32_t* d_st = ev_status;
  unsigned char* ws = nullptr;
  cudaError_t e = cudaSuccess;
  // host outputs: one device workspace, each part starting on a 256-byte boundary
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_prob = up(n * sizeof(double)), b_w = up(2 * n * sizeof(double));
  const size_t b_st = up(n * sizeof(int32_t));
  if (!dev) {
    e = cudaMallocAsync((void**)&ws, b_prob + b_w + b_st, st);
    if (e != cudaSuccess) {
      set_last_error("mem_parton_weights: workspace allocation failed");
      return e == cudaErrorMemoryAllocation ? MEM_ERR_OOM : MEM_ERR_CUDA;
    }
    d_prob = reinterpret_cast<double*>(ws);
    d_w = w_assign ? reinterpret_cast<double*>(ws + b_prob) : nullptr;
    d_st = ev_status ? reinterpret_cast<int32_t*>(ws + b_prob + b_w) : nullptr;
  }
  k_parton_tt<<<grid, PARTON_THREADS, 0, st>>>(events->d_recs, n, P, pref, d_prob, d_w, d_st);
  e = cudaGetLastError();
  if (!dev) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(prob, d_prob, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && w_assign)
      e = cudaMemcpyAsync(w_assign, d_w, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ev_status)
      e = cudaMemcpyAsync(ev_status, d_st, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    set_last_error((std::string("mem_parton_weights: ") + cudaGetErrorString(e)).c_str());
    return MEM_ERR_CUDA;
  }
  return MEM_OK;
}
