// mem_integrate_noalloc: the integration of mem_integrate for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where device allocation is not allowed after
// start-up, for example an online (trigger-level) event selection inside an
// experiment's data-acquisition process, which reserves all of its GPU memory
// when it starts and forbids allocations per event batch to keep latency
// predictable and the memory pool unfragmented, or a host application that
// hands this library device buffers from its own pool and does not let
// libraries call cudaMalloc. Such callers pass event records and outputs in
// device memory they own; the working memory (VEGAS grids, per-item
// constants, partial sums) comes from one fixed array in this file.
//
// The first call on a device is a set-up call: it resolves the array's device
// address, and CUDA's lazy module loading loads the kernels' module (which
// holds the array) and the kernels on their first launch, which reserves
// device memory. A caller that may not allocate later makes one small call
// per process kind it uses at start-up, before it reserves its memory pool
// and before any stream capture; later calls allocate nothing.
//
// Stack: the kernels of kinds 0-3 need at most 1024 bytes of per-thread stack
// (ptxas), within the context's default 1024-byte limit, so no launch grows
// the context's local memory; the dilepton ttH and ttbb kernels need more and
// are rejected.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mem.h"
#include "mem_internal.h"

namespace {

// Working memory of every mem_integrate_noalloc call on a device. Each GPU
// that loads the library holds MEM_NOALLOC_SCRATCH_BYTES of it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MEM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
// Device address of g_noalloc_scratch per device. In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached here.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_lock;

mem_status bad(const std::string& m) {
  mem::set_last_error(m.c_str());
  return MEM_ERR_INVALID_ARG;
}

mem_status cuda_bad(cudaError_t e, const char* what) {
  const std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  mem::set_last_error(m.c_str());
  return MEM_ERR_CUDA;
}

// True for plain device memory of device `dev` (not host, pinned, managed or
// another GPU's memory): the kernels of this entry point read and write these
// pointers directly and copy nothing.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" mem_status mem_integrate_noalloc(const mem_process_desc* desc, const mem_tf_desc* tf,
                                            const float* records, int64_t n_events,
                                            uint64_t n_points, uint64_t seed,
                                            uint64_t event_id_base, double* prob, double* err,
                                            int32_t* ev_status, void* stream) {
  using namespace mem;
  if (!desc || !tf || !records || !prob || !err) return bad("NULL argument");
  const int kind = desc->kind;
  const int d = dims_of(kind), np = nperm_of(kind);
  if (d < 0 || desc->reserved != 0) return bad("unknown process kind or reserved != 0");
  // the dilepton ttH and ttbb kernels raise the context's per-thread stack limit before
  // their first launch, which reserves device memory: not this entry point's contract
  if (kind == PROC_TTH || kind == PROC_TTBB)
    return bad("dilepton ttH and ttbb need mem_integrate (their kernels reserve a larger stack)");
  const double v[] = {desc->sqrt_s, desc->mz, desc->wz, desc->mw, desc->ww, desc->mt,
                      desc->wt, desc->alpha, desc->sw2, desc->alpha_s};
  for (double x : v)
    if (!(x > 0.0) || !std::isfinite(x)) return bad("masses, widths, couplings and sqrt_s must be positive");
  if (!(desc->sw2 < 1.0)) return bad("sw2 must be < 1");
  for (int t = 0; t < 3; ++t)
    if (!(desc->pdf_A[t] > 0.0) || !std::isfinite(desc->pdf_a[t]) || !(desc->pdf_b[t] >= 0.0))
      return bad("PDF parameters need A > 0, finite a, b >= 0");
  if ((kind == PROC_DY || kind == PROC_W) &&
      !(tf->lep_rel > 0 && tf->window_k > 0 && tf->lep_rel * tf->window_k < 1))
    return bad("lepton TF needs lep_rel > 0, window_k > 0, lep_rel*window_k < 1");
  if ((kind == PROC_W || kind == PROC_TTBAR) && !(tf->met_sigma > 0 && tf->met_box_k > 0))
    return bad("MET TF needs met_sigma > 0 and met_box_k > 0");
  if ((kind == PROC_TTBAR || kind == PROC_TTDL || kind == PROC_TTH || kind == PROC_TTBB) &&
      !(tf->jet_core > 0 && tf->jet_tail > 0 && tf->jet_tail_w >= 0 && tf->jet_tail_w <= 1 &&
        tf->jet_lo_div > 1 && tf->jet_hi_mul > 1))
    return bad("invalid jet TF parameters");
  if (n_events < 1 || n_events > ((int64_t)1 << 31)) return bad("n_events out of range");
  if (n_points > ((uint64_t)1 << 32)) return bad("n_points above 2^32 per item");
  // default plan of mem_integrate: 5 adaptation iterations of min(2^14, n/8) points
  const int iters = 5;
  const uint64_t na = n_points / 8 < 16384 ? n_points / 8 : 16384;
  if (na < 1 || n_points < (uint64_t)iters * na + 2) return bad("n_points too small (need >= 16)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_bad(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return bad("device index above the supported 64");
  if (!on_device(records, dev)) return bad("records must be device memory of the current device");
  if (!on_device(prob, dev) || !on_device(err, dev) || (ev_status && !on_device(ev_status, dev)))
    return bad("prob, err and ev_status must be device memory of the current device (this entry "
               "point copies nothing)");

  const int64_t n_items = n_events * np;
  const uint32_t n_main = (uint32_t)(n_points - (uint64_t)iters * na);
  const uint32_t cp = chunk_points(kind);
  const uint32_t cpi = (n_main + cp - 1) / cp;
  const size_t grid_bytes = up256((size_t)n_items * d * NG * sizeof(GridBin));
  const size_t cache_bytes = up256((size_t)n_items * cache_size(kind));
  const size_t slot_bytes = up256((size_t)n_items * cpi * sizeof(Slot));
  const size_t need = grid_bytes + cache_bytes + slot_bytes;
  if (need > (size_t)MEM_NOALLOC_SCRATCH_BYTES)
    return bad("needs " + std::to_string(need) + " bytes of working memory, above the fixed " +
               std::to_string((size_t)MEM_NOALLOC_SCRATCH_BYTES) +
               " bytes of mem_integrate_noalloc: use fewer events or points per call");

  void* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_scratch_lock);
    if (!g_scratch_addr[dev]) {
      // first call on this device (with it current): resolve the array's device address
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_bad(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  unsigned char* ws = reinterpret_cast<unsigned char*>(base);
  // every region below is fully written before it is read in the same call
  // (grids and constants by the adaptation kernel, one slot per sampling CTA),
  // so nothing left by an earlier call needs clearing
  IntegrateArgs a;
  a.recs = records;
  a.n_events = n_events;
  a.n_items = n_items;
  a.P = make_proc_const_from(desc);
  a.T = make_tf_const_from(tf);
  a.seed = seed;
  a.event_id_base = event_id_base;
  a.n_iters = iters;
  a.n_adapt = (uint32_t)na;
  a.alpha = 1.5;
  a.grid_in = nullptr;
  a.idx0 = (uint32_t)((uint64_t)iters * na);
  a.n_main = n_main;
  a.chunks_per_item = cpi;
  a.grid32 = reinterpret_cast<GridBin*>(ws);
  a.caches = ws + grid_bytes;
  a.slots = reinterpret_cast<Slot*>(ws + grid_bytes + cache_bytes);
  a.phase_events = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  e = launch_integrate(kind, a, st);
  if (e == cudaSuccess)
    e = launch_final(a.slots, n_events, np, cpi, n_main, n_points, 0, a.P.prefactor, prob, err,
                     nullptr, ev_status, st);
  if (e != cudaSuccess) return cuda_bad(e, "mem_integrate_noalloc");
  return MEM_OK;
}
