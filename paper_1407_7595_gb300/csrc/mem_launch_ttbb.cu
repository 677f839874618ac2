// Kernel instantiations for the dilepton ttbb process (fixed-budget integration and
// point evaluation), and the colour matrices of its production terms.
#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>
#include <vector>

#include "mem_launch.cuh"
#include "mem_launch_config.h"
#include "mem_ttbb.cuh"

namespace mem {
namespace {

using cd = std::complex<double>;

// SU(3) generators t^a = lambda^a / 2 and structure constants f^{abc} = -2 i Tr([t^a, t^b] t^c)
struct SU3 {
  cd t[8][3][3];
  double f[8][8][8];
  SU3() {
    for (auto& a : t)
      for (auto& r : a)
        for (auto& x : r) x = 0.0;
    const cd I(0.0, 1.0);
    const double h = 0.5, r3 = 1.0 / std::sqrt(3.0);
    t[0][0][1] = t[0][1][0] = h;
    t[1][0][1] = -I * h; t[1][1][0] = I * h;
    t[2][0][0] = h; t[2][1][1] = -h;
    t[3][0][2] = t[3][2][0] = h;
    t[4][0][2] = -I * h; t[4][2][0] = I * h;
    t[5][1][2] = t[5][2][1] = h;
    t[6][1][2] = -I * h; t[6][2][1] = I * h;
    t[7][0][0] = t[7][1][1] = h * r3; t[7][2][2] = -2.0 * h * r3;
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        for (int c = 0; c < 8; ++c) {
          cd tr = 0.0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              for (int k = 0; k < 3; ++k)
                tr += (t[a][i][j] * t[b][j][k] - t[b][i][j] * t[a][j][k]) * t[c][k][i];
          f[a][b][c] = std::real(-2.0 * I * tr);
        }
  }
  // (t^{x0} t^{x1} ...)_{ij}
  cd prod(const int* x, int n, int i, int j) const {
    cd M[3][3], R[3][3];
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) M[p][q] = p == q ? 1.0 : 0.0;
    for (int s = 0; s < n; ++s) {
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
          R[p][q] = 0.0;
          for (int r = 0; r < 3; ++r) R[p][q] += M[p][r] * t[x[s]][r][q];
        }
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) M[p][q] = R[p][q];
    }
    return M[i][j];
  }
};

const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// colour tensor of g g term n (the order of ttbb_amp2) at gluon colours a, b, top i,
// antitop j, b k, bbar l
cd gg_colour(const SU3& S, int n, int a, int b, int i, int j, int k, int l) {
  cd s = 0.0;
  if (n < 12) {   // A (top line) and B (b line): the three vertices in order, pair gluon c
    const bool top = n < 6;
    const int* pm = kPerm[top ? n : n - 6];
    for (int c = 0; c < 8; ++c) {
      const int idx[3] = {a, b, c};
      const int x[3] = {idx[pm[0]], idx[pm[1]], idx[pm[2]]};
      s += top ? S.prod(x, 3, i, j) * S.t[c][k][l] : S.prod(x, 3, k, l) * S.t[c][i][j];
    }
    return s;
  }
  if (n < 20) {   // C: order x, b-line order, top-line order
    const int r = n - 12, xg = r / 4, bo = (r / 2) % 2, to = r % 2;
    const int cx = xg == 0 ? a : b, cy = xg == 0 ? b : a;
    for (int c = 0; c < 8; ++c) {
      int xt[2], xb[2];
      xt[to] = cx; xt[1 - to] = c;
      xb[bo] = cy; xb[1 - bo] = c;
      s += S.prod(xt, 2, i, j) * S.prod(xb, 2, k, l);
    }
    return s;
  }
  if (n < 24) {   // D: f^{abe}, gluon e on a line with the other pair's gluon c
    const int r = n - 20, line = r / 2, o = r % 2;
    for (int e = 0; e < 8; ++e)
      for (int c = 0; c < 8; ++c) {
        if (S.f[a][b][e] == 0.0) continue;
        int x[2];
        x[o] = e; x[1 - o] = c;
        s += S.f[a][b][e] * (line == 0 ? S.prod(x, 2, i, j) * S.t[c][k][l] : S.prod(x, 2, k, l) * S.t[c][i][j]);
      }
    return s;
  }
  if (n < 32) {   // E: f^{x c e}: legs (external x, pair gluon c, joining gluon e)
    const int r = n - 24, xg = r / 4, line = (r / 2) % 2, o = r % 2;
    const int cx = xg == 0 ? a : b, cy = xg == 0 ? b : a;
    for (int c = 0; c < 8; ++c)
      for (int e = 0; e < 8; ++e) {
        if (S.f[cx][c][e] == 0.0) continue;
        int x[2];
        x[o] = cy; x[1 - o] = e;
        s += S.f[cx][c][e] * (line == 0 ? S.prod(x, 2, i, j) * S.t[c][k][l] : S.prod(x, 2, k, l) * S.t[c][i][j]);
      }
    return s;
  }
  for (int c = 0; c < 8; ++c)    // F and G: pair gluons c (top), d (b)
    for (int d = 0; d < 8; ++d) {
      const cd td = S.t[c][i][j] * S.t[d][k][l];
      if (td == 0.0) continue;
      double f = 0.0;
      for (int e = 0; e < 8; ++e) {
        switch (n) {
          case 32: f += S.f[a][b][e] * S.f[c][d][e]; break;
          case 33: f += S.f[a][c][e] * S.f[b][d][e]; break;
          case 34: f += S.f[a][d][e] * S.f[b][c][e]; break;
          case 35: f += S.f[a][b][e] * S.f[e][c][d]; break;
          case 36: f += S.f[a][c][e] * S.f[b][d][e]; break;
          default: f += S.f[b][c][e] * S.f[a][d][e]; break;
        }
      }
      s += f * td;
    }
  return s;
}

// colour tensor of q qbar term n at the quark iq, antiquark jq colours (the light line
// read from the antiquark row to the quark column: (t ...)_{jq iq})
cd qq_colour(const SU3& S, int n, int iq, int jq, int i, int j, int k, int l) {
  cd s = 0.0;
  if (n < 4) {
    const int line = n / 2, o = n % 2;
    for (int e = 0; e < 8; ++e)
      for (int c = 0; c < 8; ++c) {
        int x[2];
        x[o] = e; x[1 - o] = c;
        s += S.t[e][jq][iq] * (line == 0 ? S.prod(x, 2, i, j) * S.t[c][k][l] : S.prod(x, 2, k, l) * S.t[c][i][j]);
      }
    return s;
  }
  if (n == 4) {
    for (int e = 0; e < 8; ++e)
      for (int c = 0; c < 8; ++c)
        for (int d = 0; d < 8; ++d)
          if (S.f[e][c][d] != 0.0) s += S.t[e][jq][iq] * S.f[e][c][d] * S.t[c][i][j] * S.t[d][k][l];
    return s;
  }
  const int o = n - 5;
  for (int c = 0; c < 8; ++c)
    for (int d = 0; d < 8; ++d) {
      int x[2];
      x[o] = c; x[1 - o] = d;
      s += S.prod(x, 2, jq, iq) * S.t[c][i][j] * S.t[d][k][l];
    }
  return s;
}

std::vector<cd> colour_matrix_d(bool gg) {
  static const SU3 S;
  const int N = gg ? TTBB_NGG : TTBB_NQQ, ext = gg ? 64 : 9;
  std::vector<cd> Cm((size_t)N * ext * 81);
  for (int n = 0; n < N; ++n) {
    size_t q = (size_t)n * ext * 81;
    for (int a = 0; a < (gg ? 8 : 3); ++a)
      for (int b = 0; b < (gg ? 8 : 3); ++b)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
              for (int l = 0; l < 3; ++l)
                Cm[q++] = gg ? gg_colour(S, n, a, b, i, j, k, l) : qq_colour(S, n, a, b, i, j, k, l);
  }
  std::vector<cd> K((size_t)N * N);
  for (int n = 0; n < N; ++n)
    for (int m = 0; m < N; ++m) {
      cd s = 0.0;
      for (int q = 0; q < ext * 81; ++q) s += std::conj(Cm[(size_t)n * ext * 81 + q]) * Cm[(size_t)m * ext * 81 + q];
      K[(size_t)n * N + m] = s;
    }
  return K;
}

std::vector<float2> colour_matrix(bool gg) {
  const std::vector<cd> K = colour_matrix_d(gg);
  std::vector<float2> r(K.size());
  for (size_t q = 0; q < K.size(); ++q) r[q] = make_float2((float)K[q].real(), (float)K[q].imag());
  return r;
}

// K = sum_k u_k u_k^dagger by pivoted Cholesky (K is Hermitian positive semidefinite,
// a Gram matrix): each step takes the largest remaining diagonal element as pivot p,
// u = K[:, p] / sqrt(K[p][p]), and removes u u^dagger; it stops when every remaining
// diagonal element is below 1e-12 of the largest initial one (the numerical rank).
// Returns the rows conj(u_k) (rank x N) and the rank; rank -1 if the factors do not
// reproduce K to 1e-9 of its largest diagonal element.
struct ColourFactors {
  std::vector<float2> w;
  int rank;
};

ColourFactors colour_factors(bool gg) {
  const std::vector<cd> K = colour_matrix_d(gg);
  const int N = gg ? TTBB_NGG : TTBB_NQQ;
  std::vector<cd> A(K);
  double dmax = 0.0;
  for (int n = 0; n < N; ++n) dmax = std::max(dmax, A[(size_t)n * N + n].real());
  std::vector<std::vector<cd>> us;
  for (int k = 0; k < N; ++k) {
    int p = -1;
    double best = 1e-12 * dmax;
    for (int n = 0; n < N; ++n)
      if (A[(size_t)n * N + n].real() > best) {
        best = A[(size_t)n * N + n].real();
        p = n;
      }
    if (p < 0) break;
    const double sq = std::sqrt(best);
    std::vector<cd> u(N);
    for (int n = 0; n < N; ++n) u[n] = A[(size_t)n * N + p] / sq;
    for (int n = 0; n < N; ++n)
      for (int m = 0; m < N; ++m) A[(size_t)n * N + m] -= u[n] * std::conj(u[m]);
    us.push_back(u);
  }
  ColourFactors r;
  r.rank = (int)us.size();
  double err = 0.0;
  for (int n = 0; n < N; ++n)
    for (int m = 0; m < N; ++m) {
      cd s = 0.0;
      for (const auto& u : us) s += u[n] * std::conj(u[m]);
      err = std::max(err, std::abs(s - K[(size_t)n * N + m]));
    }
  if (!(err <= 1e-9 * dmax)) r.rank = -1;
  r.w.assign((size_t)N * N, make_float2(0.f, 0.f));
  for (size_t k = 0; k < us.size(); ++k)
    for (int m = 0; m < N; ++m) r.w[k * N + m] = make_float2((float)us[k][m].real(), (float)-us[k][m].imag());
  return r;
}

// The colour matrices' factors in constant memory: uploaded once per device (constant
// memory belongs to each device's context), at the first call that launches a
// ttbb kernel on it, before any stream capture.
cudaError_t ttbb_colour_upload() {
  static const ColourFactors ugg = colour_factors(true), uqq = colour_factors(false);
  if (ugg.rank < 1 || uqq.rank < 1) return cudaErrorInvalidValue;
  static std::mutex lock;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(lock);
  if (done[dev]) return cudaSuccess;
  const int ranks[2] = {ugg.rank, uqq.rank};
  e = cudaMemcpyToSymbol(c_ttbb_ugg, ugg.w.data(), ugg.w.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ttbb_uqq, uqq.w.data(), uqq.w.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ttbb_rank, ranks, sizeof(ranks));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// The ttbb kernels keep up to ~3 KB per thread on the stack (ptxas: see the
// stack-frame record in profiles/); raise the context's per-thread stack limit
// to 4 KB if it is lower (this reserves device memory once per context).
cudaError_t ttbb_stack() {
  size_t cur = 0;
  cudaError_t e = cudaDeviceGetLimit(&cur, cudaLimitStackSize);
  if (e == cudaSuccess && cur < 4096) e = cudaDeviceSetLimit(cudaLimitStackSize, 4096);
  return e;
}

}  // namespace

cudaError_t prepare_ttbb() {
  cudaError_t e = ttbb_stack();
  if (e == cudaSuccess) e = ttbb_colour_upload();
  return e;
}

cudaError_t launch_integrate_ttbb(const IntegrateArgs& a, cudaStream_t st) {
  cudaError_t e = prepare_ttbb();
  if (e != cudaSuccess) return e;
  return run_integrate<PhysTTBB, PPT_DL, MINB_BB, MINB_BB_MAIN>(a, st);
}
cudaError_t launch_eval_ttbb(const EvalArgs& a, cudaStream_t st) {
  cudaError_t e = prepare_ttbb();
  if (e != cudaSuccess) return e;
  return run_eval<PhysTTBB>(a, st);
}
size_t cache_size_ttbb() { return cache_bytes<PhysTTBB>(); }

}  // namespace mem

#include "mem_batch.cuh"

namespace mem {
// adaptive rounds; prepare_ttbb() must have run on this device (outside any capture)
cudaError_t launch_batch_ttbb(const BatchArgs& b, cudaStream_t st) {
  return run_batch<PhysTTBB, MINB_BB>(b, st);
}
}  // namespace mem

extern "C" mem_status mem_ttbb_colour_matrices(float* kgg, float* kqq) {
  if (!kgg || !kqq) return MEM_ERR_INVALID_ARG;
  const std::vector<float2> a = mem::colour_matrix(true), b = mem::colour_matrix(false);
  for (size_t q = 0; q < a.size(); ++q) {
    kgg[2 * q] = a[q].x;
    kgg[2 * q + 1] = a[q].y;
  }
  for (size_t q = 0; q < b.size(); ++q) {
    kqq[2 * q] = b[q].x;
    kqq[2 * q + 1] = b[q].y;
  }
  return MEM_OK;
}

extern "C" mem_status mem_ttbb_colour_factors(float* ugg, float* uqq, int32_t* ranks) {
  if (!ugg || !uqq || !ranks) return MEM_ERR_INVALID_ARG;
  const mem::ColourFactors a = mem::colour_factors(true), b = mem::colour_factors(false);
  if (a.rank < 1 || b.rank < 1) return MEM_ERR_INVALID_ARG;
  for (size_t q = 0; q < a.w.size(); ++q) {
    ugg[2 * q] = a.w[q].x;
    ugg[2 * q + 1] = a.w[q].y;
  }
  for (size_t q = 0; q < b.w.size(); ++q) {
    uqq[2 * q] = b.w[q].x;
    uqq[2 * q + 1] = b.w[q].y;
  }
  ranks[0] = a.rank;
  ranks[1] = b.rank;
  return MEM_OK;
}
