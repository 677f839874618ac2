// Points per thread and launch bounds of each process's sampling kernels, chosen
// by measurement on GB300 (shared by the parametric- and tabulated-PDF builds).
#pragma once

namespace mem {

constexpr int PPT_DY = 16;       // frozen-grid points per thread (Drell-Yan): 4,096 per CTA
constexpr int PPT_W = 64;        // frozen-grid points per thread (W): 16,384 per CTA
constexpr int MINB_W = 5;        // adaptation and round kernels: 5 CTAs of 256 threads per SM (<= 51 registers)
constexpr int MINB_W_MAIN = 6;   // frozen-grid kernel: 6 CTAs per SM (<= 42 registers, 4 bytes of spill)
constexpr int PPT_TT = 16;       // frozen-grid points per thread (ttbar): 4,096 per CTA
constexpr int MINB_TT = 2;       // adaptation and round kernels: <= 128 registers, no spills
constexpr int MINB_TT_MAIN = 3;  // frozen-grid kernel: <= 80 registers (20 bytes of spill), 24 warps/SM

constexpr int PPT_DL = 16;       // frozen-grid points per thread (dilepton ttbar): 4,096 per CTA
constexpr int MINB_DL = 4;       // adaptation kernel: 4 CTAs of 256 threads per SM (<= 64 registers)
constexpr int MINB_DL_MAIN = 5;  // frozen-grid kernel: 5 CTAs per SM (<= 48 registers): the double-float
                                 // solver is latency-bound and occupancy pays for the spills (measured
                                 // against 1/2, 2/2-4, 3/4); the stack stays <= 1024 bytes, within the
                                 // default per-thread limit (5/6 would exceed it)
constexpr int MINB_TH = 3;       // dilepton ttH adaptation kernel: 3 CTAs per SM
constexpr int MINB_TH_MAIN = 4;  // dilepton ttH frozen-grid kernel: 4 CTAs per SM (measured against
                                 // 1/2, 2/2, 2/3)
constexpr int MINB_BB = 1;       // dilepton ttbb adaptation kernel: one CTA per SM (its colour forms
constexpr int MINB_BB_MAIN = 2;  // need the registers: 2/2, 2/3 and 3/4 measured slower)


}  // namespace mem
