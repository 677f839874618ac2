// Host-side interface between the C ABI (mem_api.cu) and the per-process
// kernel launchers (mem_launch_*.cu). Internal to libmem.so.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mem.h"
#include "mem_common.cuh"
#include "mem_physics.cuh"

constexpr uint32_t MAGIC_PROC = 0x4D454D50u;  // "MEMP"
constexpr uint32_t MAGIC_EVT = 0x4D454D45u;   // "MEME"

// Library-owned handles (opaque to callers).
struct mem_process {
  uint32_t magic;
  mem_process_desc desc;
  mem::ProcConst pc;
  float4* d_pdf_grid;   // device copy of an attached PDF table (or nullptr)
};

struct mem_events {
  uint32_t magic;
  int32_t kind;
  int64_t n;
  int device;
  float* d_recs;
};

namespace mem {
struct FlowW;
struct FlowB;
}  // namespace mem

constexpr uint32_t MAGIC_FLOW = 0x4D454D46u;  // "MEMF"

// Learned-sampler parameters (mem_flow.cu).
struct mem_flow {
  uint32_t magic;
  int device;
  mem::FlowW* W;      // FP32 master
  mem::FlowB* B;      // BF16 operands
  mem::FlowW* m;      // Adam first moment
  mem::FlowW* v;      // Adam second moment
  float* grad;        // FlowW-shaped gradient accumulator
  int64_t step;
};

void mem_flow_release(mem_flow* f);

namespace mem {

// Poll limit of the training kernel's tensor-core waits on the current device.
cudaError_t set_train_wait_limit(uint32_t polls);

struct IntegrateArgs {
  const float* recs;        // device, n_events x REC
  int64_t n_events, n_items;
  ProcConst P;
  TFConst T;
  uint64_t seed, event_id_base;
  int n_iters;              // adaptation iterations
  uint32_t n_adapt;         // points per item per adaptation iteration
  double alpha;
  const double* grid_in;    // device d x (NG+1) or nullptr
  uint32_t idx0;            // first point index of the frozen-grid phase
  uint32_t n_main;          // frozen-grid points per item
  uint32_t chunks_per_item;
  uint32_t strat_k = 0;     // stratified frozen-grid phase: points per hypercube (0 = plain)
  uint32_t strat_ns = 0;    // hypercubes per dimension
  uint32_t strat_cubes = 0; // hypercubes per item (strat_ns^D)
  uint32_t cubes_per_thread = 0;
  GridBin* grid32;          // device n_items x D x NG
  void* caches;             // device n_items x sizeof(Phys::Cache): per-item constants
  Slot* slots;              // device n_items x chunks_per_item
  cudaEvent_t* phase_events;  // optional: 4 events (before adapt, main, final; after final)
};

struct EvalArgs {
  const float* rec;         // device, one record
  int perm;
  ProcConst P;
  TFConst T;
  uint64_t seed;
  uint32_t event_id, point0;
  int64_t n;
  const GridBin* gb;        // device D x NG
  double* w_out;            // device
};

// Points per CTA of the frozen-grid kernel for a process kind.
uint32_t chunk_points(int kind);
int dims_of(int kind);
int nperm_of(int kind);

cudaError_t launch_integrate(int kind, const IntegrateArgs& a, cudaStream_t st);
cudaError_t launch_eval(int kind, const EvalArgs& a, cudaStream_t st);

// per-process entry points (defined in the launch translation units)
cudaError_t launch_integrate_dy(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_w(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_tt(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_ttdl(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_tth(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_ttbb(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_eval_dy(const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_w(const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_tt(const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_ttdl(const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_tth(const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_ttbb(const EvalArgs&, cudaStream_t);

// constants and error reporting shared with entry points outside mem_api.cu
ProcConst make_proc_const_from(const void* mem_process_desc_ptr);
TFConst make_tf_const_from(const void* mem_tf_desc_ptr);
void set_last_error(const char* msg);

size_t cache_size_dy();
size_t cache_size_w();
size_t cache_size_tt();
size_t cache_size_ttdl();
size_t cache_size_tth();
size_t cache_size_ttbb();
size_t cache_size(int kind);

struct BatchArgs;
cudaError_t launch_batch_dy(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_w(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_tt(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_ttdl(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_tth(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_ttbb(const BatchArgs&, cudaStream_t);
// Per-device set-up of the dilepton ttH / ttbb kernels (per-thread stack limit,
// ttbb colour matrices); host calls that may synchronise, so they run before
// any stream capture.
cudaError_t prepare_tth();
cudaError_t prepare_ttbb();
// The same with tabulated PDFs (P.pdf_grid set): kernels built for that path
// (mem_launch_grid.cu); the functions above forward to them.
cudaError_t launch_integrate_dy_grid(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_w_grid(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_integrate_tt_grid(const IntegrateArgs&, cudaStream_t);
cudaError_t launch_batch_dy_grid(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_w_grid(const BatchArgs&, cudaStream_t);
cudaError_t launch_batch_tt_grid(const BatchArgs&, cudaStream_t);

cudaError_t launch_final(const Slot* slots, int64_t n_events, int nperm, uint32_t cpi,
                         uint32_t n_main, uint64_t n_per_item, uint32_t n_cubes,
                         double prefactor, double* prob, double* err, uint64_t* n_used,
                         int32_t* status, cudaStream_t st);
// Hypercubes per dimension of the stratified phase: the largest s >= 1 with
// k s^d <= n (0 if n < k).
uint32_t strat_side(uint64_t n, int d, int k);

}  // namespace mem
