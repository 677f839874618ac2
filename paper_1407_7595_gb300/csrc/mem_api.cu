// C ABI of libmem.so (declared in include/mem.h): validation, process
// constants, device memory, launches and result transfer.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mem.h"
#include "mem_internal.h"
#include "mem_kernels.cuh"
#include "mem_launch_config.h"

namespace {

thread_local std::string g_err;

mem_status fail(mem_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

mem_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MEM_ERR_OOM : MEM_ERR_CUDA;
}

#define MEM_CK(call)                                  \
  do {                                                \
    cudaError_t e__ = (call);                         \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace mem {

uint32_t strat_side(uint64_t n, int d, int k) {
  uint64_t s = 0;
  for (;;) {  // increase while k (s+1)^d <= n
    uint64_t p = (uint64_t)k;
    for (int j = 0; j < d && p <= n; ++j) p *= s + 1;
    if (p > n) return (uint32_t)s;
    ++s;
  }
}

int dims_of(int kind) {
  return kind == PROC_DY ? 2 : kind == PROC_W ? 4 : kind == PROC_TTBAR ? 7 : kind == PROC_TTDL ? 6
       : (kind == PROC_TTH || kind == PROC_TTBB) ? 8 : -1;
}
int nperm_of(int kind) {
  return kind == PROC_TTBAR ? 24 : kind == PROC_TTDL ? 2 : (kind == PROC_TTH || kind == PROC_TTBB) ? 12
       : (kind == PROC_DY || kind == PROC_W) ? 1 : -1;
}
uint32_t chunk_points(int kind) {  // points of one frozen-grid CTA: THREADS x points per thread
  return THREADS * (uint32_t)(kind == PROC_DY ? PPT_DY
                              : kind == PROC_W ? PPT_W
                              : (kind == PROC_TTDL || kind == PROC_TTH || kind == PROC_TTBB) ? PPT_DL
                                                                        : PPT_TT);
}

cudaError_t launch_integrate(int kind, const IntegrateArgs& a, cudaStream_t st) {
  switch (kind) {
    case PROC_DY: return launch_integrate_dy(a, st);
    case PROC_W: return launch_integrate_w(a, st);
    case PROC_TTBAR: return launch_integrate_tt(a, st);
    case PROC_TTDL: return launch_integrate_ttdl(a, st);
    case PROC_TTH: return launch_integrate_tth(a, st);
    case PROC_TTBB: return launch_integrate_ttbb(a, st);
  }
  return cudaErrorInvalidValue;
}

size_t cache_size(int kind) {
  return kind == PROC_DY ? cache_size_dy()
         : kind == PROC_W ? cache_size_w()
         : kind == PROC_TTDL ? cache_size_ttdl()
         : kind == PROC_TTH ? cache_size_tth()
         : kind == PROC_TTBB ? cache_size_ttbb()
                            : cache_size_tt();
}

cudaError_t launch_eval(int kind, const EvalArgs& a, cudaStream_t st) {
  switch (kind) {
    case PROC_DY: return launch_eval_dy(a, st);
    case PROC_W: return launch_eval_w(a, st);
    case PROC_TTBAR: return launch_eval_tt(a, st);
    case PROC_TTDL: return launch_eval_ttdl(a, st);
    case PROC_TTH: return launch_eval_tth(a, st);
    case PROC_TTBB: return launch_eval_ttbb(a, st);
  }
  return cudaErrorInvalidValue;
}

__device__ __forceinline__ void neu_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

// n_cubes > 0: the slots hold stratified sums (per-cube means, per-cube variances
// of the mean), the item estimate is their sum / n_cubes and its variance / n_cubes^2.
__global__ void k_final(const Slot* __restrict__ slots, int64_t n_events, int nperm,
                        uint32_t cpi, uint32_t n_main, uint64_t n_per_item, uint32_t n_cubes,
                        double prefactor, double* __restrict__ prob, double* __restrict__ err,
                        uint64_t* __restrict__ n_used, int32_t* __restrict__ status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_events) return;
  double ms = 0, mc = 0, vs = 0, vc = 0;
  uint32_t nbad = 0;
  bool invalid = false;
  const double N = (double)n_main;
  for (int p = 0; p < nperm; ++p) {
    const Slot* sl = slots + ((uint64_t)e * nperm + p) * cpi;
    double s1 = 0, c1 = 0, s2 = 0, c2 = 0;
    for (uint32_t c = 0; c < cpi; ++c) {
      const Slot q = sl[c];
      neu_add(s1, c1, q.s1);
      neu_add(s1, c1, q.c1);
      neu_add(s2, c2, q.s2);
      neu_add(s2, c2, q.c2);
      nbad += q.n_bad & 0x7fffffffu;
      invalid |= (q.n_bad >> 31) != 0;
    }
    double mean, var;
    if (n_cubes) {
      const double M = (double)n_cubes;
      mean = (s1 + c1) / M;
      var = (s2 + c2) / (M * M);
    } else {
      mean = (s1 + c1) / N;
      var = ((s2 + c2) / N - mean * mean) / (N - 1.0);
    }
    var = var > 0.0 ? var : 0.0;
    neu_add(ms, mc, mean);
    neu_add(vs, vc, var);
  }
  prob[e] = prefactor * (ms + mc) / nperm;
  err[e] = prefactor * sqrt(vs + vc) / nperm;
  if (n_used) n_used[e] = n_per_item * (uint64_t)nperm;
  if (status) status[e] = invalid ? MEM_ERR_INVALID_ARG : (nbad ? MEM_ERR_NONFINITE : MEM_OK);
}

cudaError_t launch_final(const Slot* slots, int64_t n_events, int nperm, uint32_t cpi,
                         uint32_t n_main, uint64_t n_per_item, uint32_t n_cubes,
                         double prefactor, double* prob, double* err, uint64_t* n_used,
                         int32_t* status, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n_events + 127) / 128);
  k_final<<<blocks, 128, 0, st>>>(slots, n_events, nperm, cpi, n_main, n_per_item, n_cubes,
                                  prefactor, prob, err, n_used, status);
  return cudaGetLastError();
}

// D = log10(p_S / p_B), sigma_D = sqrt((e_S/p_S)^2 + (e_B/p_B)^2) / ln 10 per event.
__global__ void k_discriminant(int64_t n, const double* __restrict__ ps, const double* __restrict__ es,
                               const double* __restrict__ pb, const double* __restrict__ eb,
                               double* __restrict__ D, double* __restrict__ eD,
                               int32_t* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = ps[i], b = pb[i];
  const bool ok = a > 0.0 && b > 0.0;
  const double ra = es[i] / a, rb = eb[i] / b;
  D[i] = ok ? log10(a / b) : CUDART_NAN;
  if (eD) eD[i] = ok ? sqrt(ra * ra + rb * rb) / 2.302585092994045684 : CUDART_NAN;
  if (status) status[i] = ok ? MEM_OK : MEM_ERR_INVALID_ARG;
}

__global__ void k_philox(const __grid_constant__ PhiloxKey key, uint32_t eid, uint32_t perm,
                         uint32_t point0, int64_t n, int d, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int b = 0; 4 * b < d; ++b) {
    const u32x4 o = philox4x32_10(point0 + (uint32_t)i, (uint32_t)b << 8, eid, perm, key);
    const uint32_t w[4] = {o.a, o.b, o.c, o.d};
    for (int j = 0; j < 4 && 4 * b + j < d; ++j) out[i * d + 4 * b + j] = u01(w[j]);
  }
}

__global__ void k_refine(int d, const double* __restrict__ hist, const double* __restrict__ gin,
                         double alpha, double* __restrict__ gout) {
  extern __shared__ __align__(16) unsigned char raw[];
  double* g = reinterpret_cast<double*>(raw);           // d x (NG+1)
  double* h = g + d * (NG + 1);                         // d x NG
  double* wk = h + d * NG;                              // d x NG
  double* cum = wk + d * NG;                            // d x (NG+1)
  double* ng = cum + d * (NG + 1);                      // d x (NG+1)
  const size_t gi = blockIdx.x;
  for (int t = threadIdx.x; t < d * (NG + 1); t += blockDim.x) g[t] = gin[gi * d * (NG + 1) + t];
  for (int t = threadIdx.x; t < d * NG; t += blockDim.x) h[t] = hist[gi * d * NG + t];
  __syncthreads();
  const int j = threadIdx.x >> 5;
  if (j < d)
    refine_dim_warp(g + j * (NG + 1), h + j * NG, wk + j * NG, cum + j * (NG + 1),
                    ng + j * (NG + 1), alpha);
  __syncthreads();
  for (int t = threadIdx.x; t < d * (NG + 1); t += blockDim.x) gout[gi * d * (NG + 1) + t] = g[t];
}

// Process constants in FP64, rounded once.
ProcConst make_proc_const(const mem_process_desc& d) {
  ProcConst P;
  std::memset(&P, 0, sizeof(P));
  P.kind = d.kind;
  const double s = d.sqrt_s * d.sqrt_s;
  P.sqrt_s = (float)d.sqrt_s;
  P.s = (float)s;
  P.mz2 = (float)(d.mz * d.mz);
  P.mz2_lo = (float)(d.mz * d.mz - (double)P.mz2);
  P.mzgz = (float)(d.mz * d.wz);
  P.mw2 = (float)(d.mw * d.mw);
  P.mwgw = (float)(d.mw * d.ww);
  P.mt2 = (float)(d.mt * d.mt);
  P.mtgt = (float)(d.mt * d.wt);
  const double e2 = 4.0 * PI_D * d.alpha;
  const double gz = std::sqrt(e2 / (d.sw2 * (1.0 - d.sw2)));
  const double Ql = -1.0, T3l = -0.5;
  const double gl[2] = {gz * (T3l - Ql * d.sw2), gz * (-Ql * d.sw2)};
  double same[3] = {0, 0, 0}, opp[3] = {0, 0, 0};
  for (int fl = 0; fl < 2; ++fl) {
    const double Qq = fl == 0 ? 2.0 / 3.0 : -1.0 / 3.0, T3q = fl == 0 ? 0.5 : -0.5;
    const double gq[2] = {gz * (T3q - Qq * d.sw2), gz * (-Qq * d.sw2)};
    const double cg = e2 * Qq * Ql;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double* acc = (a == b) ? same : opp;
        acc[0] += cg * cg;
        acc[1] += 2.0 * cg * gq[a] * gl[b];
        acc[2] += (gq[a] * gl[b]) * (gq[a] * gl[b]);
      }
  }
  for (int i = 0; i < 3; ++i) {
    P.dy_same[i] = (float)same[i];
    P.dy_opp[i] = (float)opp[i];
  }
  const double g2 = e2 / d.sw2;
  P.w_coup = (float)(g2 * g2 / 12.0);
  const double gs2 = 4.0 * PI_D * d.alpha_s;
  // ttbar: g_s^4 (g^2/2)^4 x 64 (Fierz) x 6 (W- -> q qbar': colour x 2 generations) x averages
  const double tt = gs2 * gs2 * std::pow(0.5 * g2, 4) * 64.0 * 6.0;
  P.tt_gg = (float)(tt / (4.0 * 64.0));
  P.tt_qq = (float)(tt / (4.0 * 9.0));
  // ttH: Yukawas y = m / v, v = 2 m_W / g_W; W- -> mu- nubar is 1 of the 6 channels in tt
  const double vev = 2.0 * d.mw / std::sqrt(g2);
  const double yt = d.mt / vev, yb = d.mb / vev;
  P.mh2 = (float)(d.mh * d.mh);
  P.mhgh = (float)(d.mh * d.wh);
  P.tth_c = (float)(yt * yt * 3.0 * yb * yb / 6.0);
  P.gs = (float)std::sqrt(gs2);
  P.ttbb_c = (float)(std::pow(0.5 * g2, 4) * 64.0);
  for (int t = 0; t < 3; ++t) {
    P.pdfA[t] = (float)d.pdf_A[t];
    P.pdfa[t] = (float)d.pdf_a[t];
    P.pdfb[t] = (float)d.pdf_b[t];
    P.pdf_amode[t] = d.pdf_a[t] == -0.5 ? 1 : (d.pdf_a[t] == -1.0 ? 2 : 0);
    const double b = d.pdf_b[t];
    P.pdf_bint[t] = (b >= 0.0 && b <= 16.0 && b == std::floor(b)) ? (int)b : -1;
  }
  P.pdf_std = P.pdf_amode[0] == 1 && P.pdf_amode[1] == 1 && P.pdf_amode[2] == 2 &&
              P.pdf_bint[0] == 3 && P.pdf_bint[1] == 5 && P.pdf_bint[2] == 5;
  const double tp = 2.0 * PI_D;
  if (d.kind == PROC_DY) P.prefactor = (2.0 / s) / (4.0 * tp * tp);
  else if (d.kind == PROC_W) P.prefactor = (2.0 / s) / (8.0 * tp * tp);
  else if (d.kind == PROC_TTH || d.kind == PROC_TTBB)   // eight final-state particles
    P.prefactor = (2.0 / s) * std::pow(tp, 4.0 - 24.0) / 256.0 / TTH_WEIGHT_SCALE / TTH_DEC_SCALE /
                  (double)TTH_OUT_SCALE;
  else P.prefactor = (2.0 / s) * std::pow(tp, 4.0 - 18.0) / 64.0 / TT_WEIGHT_SCALE;
  return P;
}

TFConst make_tf_const(const mem_tf_desc& t) {
  TFConst T;
  T.lep_rel = (float)t.lep_rel;
  T.window_k = (float)t.window_k;
  T.jet_core = (float)t.jet_core;
  T.jet_tail = (float)t.jet_tail;
  T.jet_tail_w = (float)t.jet_tail_w;
  T.jet_lo_div = (float)t.jet_lo_div;
  T.jet_hi_mul = (float)t.jet_hi_mul;
  T.met_sigma = (float)t.met_sigma;
  T.met_box_k = (float)t.met_box_k;
  return T;
}

ProcConst make_proc_const_from(const void* p) {
  return make_proc_const(*reinterpret_cast<const mem_process_desc*>(p));
}
TFConst make_tf_const_from(const void* p) {
  return make_tf_const(*reinterpret_cast<const mem_tf_desc*>(p));
}
void set_last_error(const char* msg) { g_err = msg; }

}  // namespace mem

using namespace mem;

namespace {

mem_status check_tf(const mem_tf_desc* tf, int kind) {
  if (!tf) return fail(MEM_ERR_INVALID_ARG, "tf is NULL");
  // ttbar processes: leptons measured exactly; dilepton ttbar: MET is the visible imbalance
  if ((kind == PROC_DY || kind == PROC_W) &&
      !(tf->lep_rel > 0 && tf->window_k > 0 && tf->lep_rel * tf->window_k < 1))
    return fail(MEM_ERR_INVALID_ARG, "lepton TF needs lep_rel > 0, window_k > 0, lep_rel*window_k < 1");
  if ((kind == PROC_W || kind == PROC_TTBAR) && !(tf->met_sigma > 0 && tf->met_box_k > 0))
    return fail(MEM_ERR_INVALID_ARG, "MET TF needs met_sigma > 0 and met_box_k > 0");
  if ((kind == PROC_TTBAR || kind == PROC_TTDL || kind == PROC_TTH || kind == PROC_TTBB) &&
      !(tf->jet_core > 0 && tf->jet_tail > 0 && tf->jet_tail_w >= 0 && tf->jet_tail_w <= 1 &&
        tf->jet_lo_div > 1 && tf->jet_hi_mul > 1))
    return fail(MEM_ERR_INVALID_ARG, "invalid jet TF parameters");
  return MEM_OK;
}

// Host grid d x 129 (FP64) -> device FP32 bins (left edge, width).
std::vector<GridBin> host_bins(const double* grid, int d) {
  std::vector<GridBin> gb((size_t)d * NG);
  for (int j = 0; j < d; ++j)
    for (int i = 0; i < NG; ++i) {
      const double a = grid ? grid[j * (NG + 1) + i] : (double)i / NG;
      const double b = grid ? grid[j * (NG + 1) + i + 1] : (double)(i + 1) / NG;
      gb[(size_t)j * NG + i] = {(float)a, (float)(b - a), (float)(1.0 - b), 0.f};
    }
  return gb;
}

bool grid_valid(const double* grid, int d) {
  for (int j = 0; j < d; ++j) {
    const double* g = grid + j * (NG + 1);
    if (g[0] != 0.0 || g[NG] != 1.0) return false;
    for (int i = 0; i < NG; ++i)
      if (!(g[i + 1] > g[i])) return false;
  }
  return true;
}

}  // namespace

extern "C" {

int32_t mem_process_dims(int32_t kind) { return dims_of(kind); }
int32_t mem_process_nperm(int32_t kind) { return nperm_of(kind); }

const char* mem_last_error(void) { return g_err.c_str(); }

mem_status mem_create_process(const mem_process_desc* desc, mem_process** out) {
  if (!desc || !out) return fail(MEM_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (dims_of(desc->kind) < 0) return fail(MEM_ERR_INVALID_ARG, "unknown process kind");
  if (desc->reserved != 0) return fail(MEM_ERR_INVALID_ARG, "reserved field must be 0");
  const double v[] = {desc->sqrt_s, desc->mz, desc->wz, desc->mw, desc->ww, desc->mt,
                      desc->wt, desc->alpha, desc->sw2, desc->alpha_s};
  for (double x : v)
    if (!(x > 0.0) || !std::isfinite(x)) return fail(MEM_ERR_INVALID_ARG, "masses, widths, couplings and sqrt_s must be positive");
  if (!(desc->sw2 < 1.0)) return fail(MEM_ERR_INVALID_ARG, "sw2 must be < 1");
  if (desc->kind == PROC_TTH && !(desc->mh > 0.0 && desc->wh > 0.0 && desc->mb > 0.0 &&
                                  std::isfinite(desc->mh + desc->wh + desc->mb)))
    return fail(MEM_ERR_INVALID_ARG, "ttH needs mh, wh, mb > 0");
  for (int t = 0; t < 3; ++t)
    if (!(desc->pdf_A[t] > 0.0) || !std::isfinite(desc->pdf_a[t]) || !(desc->pdf_b[t] >= 0.0))
      return fail(MEM_ERR_INVALID_ARG, "PDF parameters need A > 0, finite a, b >= 0");
  mem_process* p = new mem_process;
  p->magic = MAGIC_PROC;
  p->desc = *desc;
  p->pc = make_proc_const(*desc);
  p->d_pdf_grid = nullptr;
  *out = p;
  return MEM_OK;
}

mem_status mem_process_set_pdf_grid(mem_process* proc, const float* table, int32_t n_x,
                                    int32_t n_q, double lnx_min, double lnx_max,
                                    double lnq_min, double lnq_max) {
  if (!proc || proc->magic != MAGIC_PROC) return fail(MEM_ERR_INVALID_ARG, "invalid process handle");
  if (!table) {  // back to the parametric set
    if (proc->d_pdf_grid) cudaFree(proc->d_pdf_grid);
    proc->d_pdf_grid = nullptr;
    proc->pc.pdf_grid = nullptr;
    return MEM_OK;
  }
  if (n_x < 2 || n_q < 2 || (int64_t)n_x * n_q > ((int64_t)1 << 24))
    return fail(MEM_ERR_INVALID_ARG, "PDF grid needs 2 <= n_x, n_q and n_x * n_q <= 2^24");
  const double b[] = {lnx_min, lnx_max, lnq_min, lnq_max};
  for (double v : b)
    if (!std::isfinite(v)) return fail(MEM_ERR_INVALID_ARG, "PDF grid bounds must be finite");
  if (!(lnx_min < lnx_max && lnx_max <= 0.0 && lnq_min < lnq_max))
    return fail(MEM_ERR_INVALID_ARG, "PDF grid needs lnx_min < lnx_max <= 0 and lnq_min < lnq_max");
  const size_t cells = (size_t)n_x * n_q;
  std::vector<float4> packed(cells);
  for (size_t k = 0; k < cells; ++k) {
    const float q = table[k], qb = table[cells + k], g = table[2 * cells + k];
    if (!(std::isfinite(q) && std::isfinite(qb) && std::isfinite(g) && q >= 0.f && qb >= 0.f &&
          g >= 0.f))
      return fail(MEM_ERR_INVALID_ARG, "PDF grid values must be finite and >= 0");
    packed[k] = make_float4(q, qb, g, 0.f);
  }
  float4* d = nullptr;
  MEM_CK(cudaMalloc(&d, cells * sizeof(float4)));
  cudaError_t e = cudaMemcpy(d, packed.data(), cells * sizeof(float4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "mem_process_set_pdf_grid");
  }
  if (proc->d_pdf_grid) cudaFree(proc->d_pdf_grid);
  proc->d_pdf_grid = d;
  ProcConst& P = proc->pc;
  P.pdf_grid = d;
  P.grid_nx = n_x;
  P.grid_nq = n_q;
  P.glx0 = (float)lnx_min;
  P.g_inv_hx = (float)((n_x - 1) / (lnx_max - lnx_min));
  P.glq0 = (float)lnq_min;
  P.g_inv_hq = (float)((n_q - 1) / (lnq_max - lnq_min));
  P.ln_rs = (float)std::log(proc->desc.sqrt_s);
  return MEM_OK;
}

mem_status mem_upload_events(mem_process* proc, const float* records, int64_t n_events,
                             int32_t records_on_device, void* stream, mem_events** out) {
  if (!proc || proc->magic != MAGIC_PROC || !records || !out)
    return fail(MEM_ERR_INVALID_ARG, "NULL or invalid argument");
  *out = nullptr;
  if (n_events < 1) return fail(MEM_ERR_INVALID_ARG, "n_events must be >= 1");
  if (n_events > (int64_t)1 << 31) return fail(MEM_ERR_INVALID_ARG, "n_events above 2^31");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)n_events * REC * sizeof(float);
  if (!records_on_device) {
    for (int64_t i = 0; i < n_events; ++i)
      if (records[i * REC + 27] != (float)proc->desc.kind)
        return fail(MEM_ERR_INVALID_ARG, "event " + std::to_string(i) + " is not of the process kind");
  }
  int dev = 0;
  MEM_CK(cudaGetDevice(&dev));
  float* d = nullptr;
  MEM_CK(cudaMalloc(&d, bytes));
  cudaError_t e = cudaMemcpyAsync(d, records, bytes,
                                  records_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "event upload");
  }
  mem_events* ev = new mem_events;
  ev->magic = MAGIC_EVT;
  ev->kind = proc->desc.kind;
  ev->n = n_events;
  ev->device = dev;
  ev->d_recs = d;
  *out = ev;
  return MEM_OK;
}

void mem_destroy(void* handle) {
  if (!handle) return;
  const uint32_t m = *reinterpret_cast<uint32_t*>(handle);
  if (m == MAGIC_PROC) {
    mem_process* p = reinterpret_cast<mem_process*>(handle);
    if (p->d_pdf_grid) cudaFree(p->d_pdf_grid);
    p->magic = 0;
    delete p;
  } else if (m == MAGIC_EVT) {
    mem_events* e = reinterpret_cast<mem_events*>(handle);
    cudaFree(e->d_recs);
    e->magic = 0;
    delete e;
  } else if (m == MAGIC_FLOW) {  // learned-sampler parameters
    mem_flow_release(reinterpret_cast<mem_flow*>(handle));
  }
}

mem_status mem_integrate(const mem_events* ev, const mem_process* proc, const mem_tf_desc* tf,
                         uint64_t n_points, uint64_t seed, const mem_opts* opts, double* prob,
                         double* err, uint64_t* n_used, int32_t* ev_status, void* stream) {
  if (!ev || ev->magic != MAGIC_EVT || !proc || proc->magic != MAGIC_PROC || !prob || !err)
    return fail(MEM_ERR_INVALID_ARG, "NULL or invalid handle/output");
  if (ev->kind != proc->desc.kind) return fail(MEM_ERR_INVALID_ARG, "events were uploaded for another process kind");
  const int kind = proc->desc.kind;
  mem_status s = check_tf(tf, kind);
  if (s != MEM_OK) return s;
  const int d = dims_of(kind), np = nperm_of(kind);
  int iters = opts ? opts->n_adapt_iters : 5;
  if (iters < 0 || iters > 64) return fail(MEM_ERR_INVALID_ARG, "n_adapt_iters out of range [0, 64]");
  if (opts && opts->flow_guided != 0) return fail(MEM_ERR_INVALID_ARG, "flow_guided must be 0");
  if (opts && opts->reserved1 != 0) return fail(MEM_ERR_INVALID_ARG, "reserved1 must be 0");
  const int strat_k = opts ? opts->strat_points : 0;
  if (strat_k == 1 || strat_k < 0 || strat_k > 64)
    return fail(MEM_ERR_INVALID_ARG, "strat_points must be 0 or in [2, 64]");
  if (strat_k && opts->target_rel_err > 0.0)
    return fail(MEM_ERR_INVALID_ARG, "stratified sampling needs the fixed-budget mode");
  if (opts && opts->target_rel_err > 0.0) {
    // adaptive budget: the batched schedule with this one event set
    const mem_events* evs[1] = {ev};
    const mem_process* prs[1] = {proc};
    const mem_tf_desc* tfs[1] = {tf};
    return mem_integrate_batch(1, evs, prs, tfs, seed, opts, prob, err, n_used, ev_status, stream);
  }
  uint64_t na = opts && opts->adapt_points ? opts->adapt_points : (n_points / 8 < 16384 ? n_points / 8 : 16384);
  if (iters == 0) na = 0;
  if (n_points > ((uint64_t)1 << 32)) return fail(MEM_ERR_INVALID_ARG, "n_points above 2^32 per item");
  if (iters > 0 && na < 1) return fail(MEM_ERR_INVALID_ARG, "adaptation needs >= 1 point per iteration");
  if (n_points < (uint64_t)iters * na + 2)
    return fail(MEM_ERR_INVALID_ARG, "n_points too small for the adaptation plan (need > iters*adapt_points + 1)");
  const double alpha = opts && opts->alpha > 0.0 ? opts->alpha : 1.5;
  const uint64_t eid_base = opts ? opts->event_id_base : 0;
  if (opts && opts->grid_in && !grid_valid(opts->grid_in, d))
    return fail(MEM_ERR_INVALID_ARG, "grid_in must have edges 0 = x0 < x1 < ... < x128 = 1 per dimension");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n_items = ev->n * np;
  const uint32_t n_main = (uint32_t)(n_points - (uint64_t)iters * na);
  const uint32_t cp = chunk_points(kind);
  uint32_t cpi = (n_main + cp - 1) / cp;
  uint32_t ns = 0, n_cubes = 0, cubes_pt = 0;
  uint64_t n_per_item = n_points;
  if (strat_k) {
    ns = strat_side(n_main, d, strat_k);
    if (ns == 0) return fail(MEM_ERR_INVALID_ARG, "stratified phase has fewer points than strat_points");
    uint64_t m = 1;
    for (int j = 0; j < d; ++j) m *= ns;
    n_cubes = (uint32_t)m;
    const uint32_t ppt = cp / THREADS;
    cubes_pt = ppt / (uint32_t)strat_k > 0 ? ppt / (uint32_t)strat_k : 1;
    const uint32_t cpc = cubes_pt * THREADS;
    cpi = (n_cubes + cpc - 1) / cpc;
    n_per_item = (uint64_t)iters * na + (uint64_t)strat_k * m;
  }

  IntegrateArgs a;
  a.recs = ev->d_recs;
  a.n_events = ev->n;
  a.n_items = n_items;
  a.P = proc->pc;
  a.T = make_tf_const(*tf);
  a.seed = seed;
  a.event_id_base = eid_base;
  a.n_iters = iters;
  a.n_adapt = (uint32_t)na;
  a.alpha = alpha;
  a.idx0 = (uint32_t)((uint64_t)iters * na);
  a.n_main = n_main;
  a.chunks_per_item = cpi;
  a.strat_k = (uint32_t)strat_k;
  a.strat_ns = ns;
  a.strat_cubes = n_cubes;
  a.cubes_per_thread = cubes_pt;
  a.phase_events = opts ? reinterpret_cast<cudaEvent_t*>(opts->phase_events) : nullptr;

  const bool dev_out = is_device_ptr(prob);
  const size_t grid_bytes = (size_t)n_items * d * NG * sizeof(GridBin);
  const size_t slot_bytes = (size_t)n_items * cpi * sizeof(Slot);
  const size_t out_bytes = dev_out ? 0 : (size_t)ev->n * (2 * sizeof(double) + sizeof(uint64_t) + sizeof(int32_t));
  const size_t gin_bytes = opts && opts->grid_in ? (size_t)d * (NG + 1) * sizeof(double) : 0;
  unsigned char* ws = nullptr;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t out_each = dev_out ? 0 : up(ev->n * sizeof(double)) * 3 + up(ev->n * sizeof(int32_t));
  const size_t cache_total = (size_t)n_items * cache_size(kind);
  const size_t total = up(grid_bytes) + up(slot_bytes) + out_each + up(gin_bytes) + up(cache_total);
  (void)out_bytes;
  MEM_CK(cudaMallocAsync((void**)&ws, total, st));
  size_t off = 0;
  auto take = [&](size_t b) {
    unsigned char* p = ws + off;
    off += (b + 255) & ~(size_t)255;
    return p;
  };
  a.grid32 = reinterpret_cast<GridBin*>(take(grid_bytes));
  a.slots = reinterpret_cast<Slot*>(take(slot_bytes));
  a.caches = take(cache_total);
  double* o_prob = prob;
  double* o_err = err;
  uint64_t* o_used = n_used;
  int32_t* o_st = ev_status;
  if (!dev_out) {
    o_prob = reinterpret_cast<double*>(take(ev->n * sizeof(double)));
    o_err = reinterpret_cast<double*>(take(ev->n * sizeof(double)));
    o_used = reinterpret_cast<uint64_t*>(take(ev->n * sizeof(uint64_t)));
    o_st = reinterpret_cast<int32_t*>(take(ev->n * sizeof(int32_t)));
  }
  a.grid_in = nullptr;
  cudaError_t e = cudaSuccess;
  if (gin_bytes) {
    double* g = reinterpret_cast<double*>(take(gin_bytes));
    e = cudaMemcpyAsync(g, opts->grid_in, gin_bytes, cudaMemcpyHostToDevice, st);
    a.grid_in = g;
  }
  if (e == cudaSuccess) e = launch_integrate(kind, a, st);
  if (e == cudaSuccess && a.phase_events) e = cudaEventRecord(a.phase_events[2], st);
  if (e == cudaSuccess)
    e = launch_final(a.slots, ev->n, np, cpi, n_main, n_per_item, n_cubes, proc->pc.prefactor,
                     o_prob, o_err, o_used, o_st, st);
  if (e == cudaSuccess && a.phase_events) e = cudaEventRecord(a.phase_events[3], st);
  if (e == cudaSuccess && !dev_out) {
    e = cudaMemcpyAsync(prob, o_prob, ev->n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err, o_err, ev->n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n_used) e = cudaMemcpyAsync(n_used, o_used, ev->n * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ev_status) e = cudaMemcpyAsync(ev_status, o_st, ev->n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  }
  cudaError_t e2 = cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && !dev_out) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "mem_integrate");
  return MEM_OK;
}

mem_status mem_eval_points(const mem_events* ev, const mem_process* proc, const mem_tf_desc* tf,
                           int64_t event_index, int32_t perm, uint64_t seed, uint64_t point0,
                           int64_t n, const double* grid, double* w_out, void* stream) {
  if (!ev || ev->magic != MAGIC_EVT || !proc || proc->magic != MAGIC_PROC || !w_out)
    return fail(MEM_ERR_INVALID_ARG, "NULL or invalid handle/output");
  if (ev->kind != proc->desc.kind) return fail(MEM_ERR_INVALID_ARG, "process kind mismatch");
  const int kind = proc->desc.kind;
  mem_status s = check_tf(tf, kind);
  if (s != MEM_OK) return s;
  if (event_index < 0 || event_index >= ev->n) return fail(MEM_ERR_INVALID_ARG, "event_index out of range");
  if (perm < 0 || perm >= nperm_of(kind)) return fail(MEM_ERR_INVALID_ARG, "perm out of range");
  if (n < 1 || point0 + (uint64_t)n > ((uint64_t)1 << 32)) return fail(MEM_ERR_INVALID_ARG, "bad point range");
  const int d = dims_of(kind);
  if (grid && !grid_valid(grid, d)) return fail(MEM_ERR_INVALID_ARG, "invalid grid");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<GridBin> gb = host_bins(grid, d);
  const bool dev_out = is_device_ptr(w_out);
  const size_t gbytes = gb.size() * sizeof(GridBin);
  unsigned char* ws = nullptr;
  MEM_CK(cudaMallocAsync((void**)&ws, gbytes + (dev_out ? 0 : n * sizeof(double)) + 256, st));
  GridBin* dgb = reinterpret_cast<GridBin*>(ws);
  double* dw = dev_out ? w_out : reinterpret_cast<double*>(ws + ((gbytes + 255) & ~(size_t)255));
  cudaError_t e = cudaMemcpyAsync(dgb, gb.data(), gbytes, cudaMemcpyHostToDevice, st);
  EvalArgs a;
  a.rec = ev->d_recs + event_index * REC;
  a.perm = perm;
  a.P = proc->pc;
  a.T = make_tf_const(*tf);
  a.seed = seed;
  a.event_id = (uint32_t)event_index;
  a.point0 = (uint32_t)point0;
  a.n = n;
  a.gb = dgb;
  a.w_out = dw;
  if (e == cudaSuccess) e = launch_eval(kind, a, st);
  if (e == cudaSuccess && !dev_out) e = cudaMemcpyAsync(w_out, dw, n * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "mem_eval_points");
  return MEM_OK;
}

mem_status mem_discriminant(int64_t n, const double* prob_s, const double* err_s,
                            const double* prob_b, const double* err_b, double* D, double* err_D,
                            int32_t* status, void* stream) {
  if (n < 1 || !prob_s || !err_s || !prob_b || !err_b || !D)
    return fail(MEM_ERR_INVALID_ARG, "invalid argument");
  const bool dev = is_device_ptr(D);
  const void* all[] = {prob_s, err_s, prob_b, err_b, err_D, status};
  for (const void* p : all)
    if (p && is_device_ptr(p) != dev)
      return fail(MEM_ERR_INVALID_ARG, "arrays must all be host or all be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t b8 = (size_t)n * sizeof(double), b4 = (size_t)n * sizeof(int32_t);
  const double *ps = prob_s, *es = err_s, *pb = prob_b, *eb = err_b;
  double *o = D, *oe = err_D;
  int32_t* os = status;
  unsigned char* ws = nullptr;
  cudaError_t e = cudaSuccess;
  if (!dev) {
    MEM_CK(cudaMallocAsync((void**)&ws, 6 * ((b8 + 255) & ~(size_t)255) + b4, st));
    auto part = [&](int k) { return reinterpret_cast<double*>(ws + k * ((b8 + 255) & ~(size_t)255)); };
    double* in[4] = {part(0), part(1), part(2), part(3)};
    const double* src[4] = {prob_s, err_s, prob_b, err_b};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(in[k], src[k], b8, cudaMemcpyHostToDevice, st);
    ps = in[0], es = in[1], pb = in[2], eb = in[3];
    o = part(4);
    oe = err_D ? part(5) : nullptr;
    os = status ? reinterpret_cast<int32_t*>(ws + 6 * ((b8 + 255) & ~(size_t)255)) : nullptr;
  }
  if (e == cudaSuccess) {
    k_discriminant<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ps, es, pb, eb, o, oe, os);
    e = cudaGetLastError();
  }
  if (!dev) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(D, o, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && err_D) e = cudaMemcpyAsync(err_D, oe, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, os, b4, cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mem_discriminant");
  return MEM_OK;
}

mem_status mem_philox_uniforms(uint64_t seed, uint64_t event_id, int32_t perm, uint64_t point0,
                               int64_t n, int32_t d, float* out, void* stream) {
  if (!out || n < 1 || d < 1 || d > MAXD || perm < 0 || point0 + (uint64_t)n > ((uint64_t)1 << 32))
    return fail(MEM_ERR_INVALID_ARG, "invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev_out = is_device_ptr(out);
  float* buf = out;
  if (!dev_out) MEM_CK(cudaMallocAsync((void**)&buf, (size_t)n * d * sizeof(float), st));
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(philox_key(seed), (uint32_t)event_id, (uint32_t)perm,
                                                        (uint32_t)point0, n, d, buf);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !dev_out) {
    e = cudaMemcpyAsync(out, buf, (size_t)n * d * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "mem_philox_uniforms");
  return MEM_OK;
}

mem_status mem_vegas_refine(int32_t n_grids, int32_t d, const double* hist, const double* grid_in,
                            double alpha, double* grid_out) {
  if (n_grids < 1 || d < 1 || d > MAXD || !hist || !grid_in || !grid_out || !(alpha > 0))
    return fail(MEM_ERR_INVALID_ARG, "invalid argument");
  const size_t gb = (size_t)n_grids * d * (NG + 1) * sizeof(double);
  const size_t hb = (size_t)n_grids * d * NG * sizeof(double);
  double *dg = nullptr, *dh = nullptr, *do_ = nullptr;
  MEM_CK(cudaMalloc(&dg, gb));
  cudaError_t e = cudaMalloc(&dh, hb);
  if (e == cudaSuccess) e = cudaMalloc(&do_, gb);
  if (e == cudaSuccess) e = cudaMemcpy(dg, grid_in, gb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dh, hist, hb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const size_t smem = (size_t)d * (3 * (NG + 1) + 2 * NG) * sizeof(double);
    e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      k_refine<<<n_grids, 32 * d, smem>>>(d, dh, dg, alpha, do_);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(grid_out, do_, gb, cudaMemcpyDeviceToHost);
  cudaFree(dg);
  cudaFree(dh);
  cudaFree(do_);
  if (e != cudaSuccess) return cuda_fail(e, "mem_vegas_refine");
  return MEM_OK;
}

}  // extern "C"
