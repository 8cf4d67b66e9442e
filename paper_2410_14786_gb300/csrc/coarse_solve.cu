// Coarse solve u_c = A_c^-1 r_c on the GPU from the supernodal factorisation
// of coarse_sparse.cpp (float64), and the same sweeps for the sparse local
// solver's interior solves t = A_II^-1 r over the forest of all subdomains'
// factors (per-level and block forms below; the mixed forms sweep with
// float32 coefficients).
//
// Vectors r' (forward right-hand side) and y (forward result) are kept in
// elimination order, so the pivots of every supernode are contiguous.
// Forward sweep, supernodes by increasing height (leaves first); for a node t
// with pivots P and update set U, [y_P; c_t] = [L_PP^-1 ; M] r'_P, and the
// contributions c_t are subtracted from r'_U. Backward sweep, by decreasing
// height: u_P = [L_PP^-T , -M^T] [y_P ; u_U].
//
// Every output value of a level is one warp unit: a row of L_PP^-1 (lower
// triangular: only its nonzero part is read), all contributions of the
// level to one later dof (its M rows summed in a fixed order, so results are
// reproducible), or a row of the backward matrix. All units of a level run
// at once across the GPU. The solve is one persistent cooperative kernel:
// levels are separated by grid-wide barriers whose waits are bounded; on
// timeout a block records BDDC_ERR_TIMEOUT and all blocks leave at their next
// barrier. Values written by other blocks are read through L2 (__ldcg).
//
// One right-hand side takes the gather form (k_coarse_sweeps): at one column
// the sweeps are bound by chains of dependent memory round trips, not by
// bytes, so every output value becomes one dot product with an explicit
// operand index per coefficient, stored in the order the warps consume them.
// The coefficients and indices are constant, so a warp loads the next batch
// of them while it waits for the operand values of the current one, and
// across each grid barrier: after a barrier only the operand loads remain.
// The contributions to a receiving dof are one contiguous dot, r' is never
// permuted (an operand that no earlier level has updated is read from r_c in
// dof order), and the units of each level are assigned to warps on the host,
// longest first to the least-loaded warp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.hpp"
#include "kernels.cuh"

namespace bddc {

namespace {

constexpr int kThreads = 1024;


struct CoarseArgs {
  const CNodeDev* nodes;
  const CUnit* units;
  const CContrib* list;      // contributions of the receiving units
  const int32_t* upd;        // update-set dofs
  const int32_t* order;      // position -> dof
  const int32_t* lvl;        // unit offsets [L+1 forward][L+1 backward], then n_c
  const double* F;
  const double* B;
  const double* r;           // r_c (dof order)
  double* rp;                // r' (elimination order)
  double* y;                 // y (elimination order)
  double* u;                 // u_c (dof order)
  unsigned int* bar;         // [0] barrier arrivals
  int32_t* err;
  int levels, nrhs;
  unsigned int bar_extra;    // arrivals a barrier waits for beyond the grid (0; > 0 only to test the waits)
  long long bar_cycles;      // limit of one barrier wait, clock cycles
};

// Grid-wide barrier; false when a wait ran out (here or in another block).
// bar counts arrivals since the launch (zeroed before it): the k-th barrier
// of a launch releases at k * gridDim.x arrivals, so no block resets it.
// Ordering: the block's writes precede thread 0's release increment (block
// barrier, then red.release at GPU scope); thread 0's acquire load of the
// final count precedes the block's later reads (then the block barrier).
__device__ bool grid_sync(unsigned int* bar, int32_t* err, unsigned int& epoch, unsigned int extra,
                          long long limit) {
  __shared__ int ok;
  const unsigned int target = ++epoch * gridDim.x + extra;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const long long t0 = clock64();
    for (;;) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (*(volatile int32_t*)err == BDDC_ERR_TIMEOUT || clock64() - t0 > limit) {
        atomicExch(err, BDDC_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    if (*(volatile int32_t*)err == BDDC_ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum_j row[j] * x[j * nrhs + k] over j in [j0, j1), one warp. Four
// elements per lane are loaded before they are used, so a row costs about
// (j1 - j0) / 128 rounds of memory latency instead of one per 32 elements.
__device__ __forceinline__ double warp_dot(const double* __restrict__ row, const double* x, int j0, int j1,
                                           int nrhs, int k, int lane) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int j = j0 + lane; j < j1; j += 128) {
    const bool b1 = j + 32 < j1, b2 = j + 64 < j1, b3 = j + 96 < j1;
    const double r0 = __ldg(&row[j]);
    const double r1 = b1 ? __ldg(&row[j + 32]) : 0.0;
    const double r2 = b2 ? __ldg(&row[j + 64]) : 0.0;
    const double r3 = b3 ? __ldg(&row[j + 96]) : 0.0;
    const double x0 = __ldcg(&x[(int64_t)j * nrhs + k]);
    const double x1 = b1 ? __ldcg(&x[(int64_t)(j + 32) * nrhs + k]) : 0.0;
    const double x2 = b2 ? __ldcg(&x[(int64_t)(j + 64) * nrhs + k]) : 0.0;
    const double x3 = b3 ? __ldcg(&x[(int64_t)(j + 96) * nrhs + k]) : 0.0;
    s0 = fma(r0, x0, s0);
    s1 = fma(r1, x1, s1);
    s2 = fma(r2, x2, s2);
    s3 = fma(r3, x3, s3);
  }
  return warp_sum((s0 + s1) + (s2 + s3));
}

// The same with x gathered: x[idx[j]] (the backward sweep's u_U).
__device__ __forceinline__ double warp_dot_gather(const double* __restrict__ row, const double* x,
                                                  const int32_t* __restrict__ idx, int n, int nrhs, int k,
                                                  int lane) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int j = lane; j < n; j += 128) {
    const bool b1 = j + 32 < n, b2 = j + 64 < n, b3 = j + 96 < n;
    const int i0 = __ldg(&idx[j]);
    const int i1 = b1 ? __ldg(&idx[j + 32]) : 0;
    const int i2 = b2 ? __ldg(&idx[j + 64]) : 0;
    const int i3 = b3 ? __ldg(&idx[j + 96]) : 0;
    const double r0 = __ldg(&row[j]);
    const double r1 = b1 ? __ldg(&row[j + 32]) : 0.0;
    const double r2 = b2 ? __ldg(&row[j + 64]) : 0.0;
    const double r3 = b3 ? __ldg(&row[j + 96]) : 0.0;
    const double x0 = __ldcg(&x[(int64_t)i0 * nrhs + k]);
    const double x1 = b1 ? __ldcg(&x[(int64_t)i1 * nrhs + k]) : 0.0;
    const double x2 = b2 ? __ldcg(&x[(int64_t)i2 * nrhs + k]) : 0.0;
    const double x3 = b3 ? __ldcg(&x[(int64_t)i3 * nrhs + k]) : 0.0;
    s0 = fma(r0, x0, s0);
    s1 = fma(r1, x1, s1);
    s2 = fma(r2, x2, s2);
    s3 = fma(r3, x3, s3);
  }
  return warp_sum((s0 + s1) + (s2 + s3));
}

// Several right-hand sides at once: columns k0 .. k0 + nr - 1 (nr <= kNR) of
// x (row-major, nrhs per row), accumulated into lane-partial sums s[k] with
// the matrix row read once for all of them.
constexpr int kNR = 8;
// Four elements per lane per round (as in warp_dot): out-of-range elements
// read a valid position and are weighted by zero, so all loads of a round
// are independent and in flight together.
__device__ __forceinline__ void warp_dot_multi(const double* __restrict__ row, const double* x, int j0, int j1,
                                               int nrhs, int k0, int nr, int lane, double (&s)[kNR]) {
  for (int j = j0 + lane; j < j1; j += 128) {
    double rv[4];
    const double* xp[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const bool in = j + 32 * t < j1;
      rv[t] = in ? __ldg(&row[j + 32 * t]) : 0.0;
      xp[t] = x + (int64_t)(in ? j + 32 * t : j) * nrhs + k0;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int k = 0; k < kNR; ++k)
        if (k < nr) s[k] = fma(rv[t], __ldcg(xp[t] + k), s[k]);
  }
}
__device__ __forceinline__ void warp_dot_gather_multi(const double* __restrict__ row, const double* x,
                                                      const int32_t* __restrict__ idx, int n, int nrhs, int k0,
                                                      int nr, int lane, double (&s)[kNR]) {
  for (int j = lane; j < n; j += 128) {
    double rv[4];
    int32_t ix[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const bool in = j + 32 * t < n;
      rv[t] = in ? __ldg(&row[j + 32 * t]) : 0.0;
      ix[t] = __ldg(&idx[in ? j + 32 * t : j]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double* xp = x + (int64_t)ix[t] * nrhs + k0;
#pragma unroll
      for (int k = 0; k < kNR; ++k)
        if (k < nr) s[k] = fma(rv[t], __ldcg(xp + k), s[k]);
    }
  }
}
// Warp sum of the 8 lane-partial sums, left on lanes with (lane & 3) == 0:
// that lane holds the total of column k = lane >> 2 (three halving
// exchanges, then two full ones: 9 shuffles instead of 40).
__device__ __forceinline__ double warp_sum8(double (&s)[kNR], int lane) {
#pragma unroll
  for (int o = 16, n = kNR; o >= 4; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double send = upper ? s[i] : s[i + n / 2];
      const double keep = upper ? s[i + n / 2] : s[i];
      s[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double v = s[0];
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

__device__ void forward_unit(const CoarseArgs& a, const CUnit& w, int lane, int kb, int ke) {
  const int nrhs = a.nrhs;
  if (w.kind == 0) {
    // y[pos0 + i] = sum_{j <= i} L_PP^-1[i, j] r'[pos0 + j]
    const CNodeDev nd = a.nodes[w.a];
    const double* row = a.F + nd.foff + (int64_t)w.row * nd.fld;
    const double* x = a.rp + (int64_t)nd.pos0 * nrhs;
    double* dst = a.y + (int64_t)(nd.pos0 + w.row) * nrhs;
    if (ke - kb == 1) {
      const double s = warp_dot(row, x, 0, w.row + 1, nrhs, kb, lane);
      if (lane == 0) dst[kb] = s;
      return;
    }
    for (int k0 = kb; k0 < ke; k0 += kNR) {
      const int nr = min(kNR, nrhs - k0);
      double s[kNR] = {0, 0, 0, 0, 0, 0, 0, 0};
      warp_dot_multi(row, x, 0, w.row + 1, nrhs, k0, nr, lane, s);
      const double v = warp_sum8(s, lane);
      if ((lane & 3) == 0 && (lane >> 2) < nr) dst[k0 + (lane >> 2)] = v;
    }
  } else {
    // r'[a] -= sum over the listed contributions, in list order, of
    // M_row . r'_P(node)
    double* dst = &a.rp[(int64_t)w.a * nrhs];
    if (ke - kb == 1) {
      double s = 0.0;
      for (int q = w.b; q < w.e; ++q) {
        const CContrib c = a.list[q];
        s += warp_dot(a.F + c.row_off, a.rp + (int64_t)c.x_off * nrhs, 0, c.len, nrhs, kb, lane);
      }
      if (lane == 0) dst[kb] = __ldcg(dst + kb) - s;
      return;
    }
    for (int k0 = kb; k0 < ke; k0 += kNR) {
      const int nr = min(kNR, nrhs - k0);
      double s[kNR] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int q = w.b; q < w.e; ++q) {
        const CContrib c = a.list[q];
        warp_dot_multi(a.F + c.row_off, a.rp + (int64_t)c.x_off * nrhs, 0, c.len, nrhs, k0, nr, lane, s);
      }
      const double v = warp_sum8(s, lane);
      if ((lane & 3) == 0 && (lane >> 2) < nr) {
        double* d = dst + k0 + (lane >> 2);
        *d = __ldcg(d) - v;
      }
    }
  }
}

__device__ void backward_unit(const CoarseArgs& a, const CUnit& w, int lane, int kb, int ke) {
  // u[dof of pos0 + i] = sum_{j >= i} L_PP^-T[i, j] y[pos0 + j] - sum_b M[b, i] u[upd_b]
  const int nrhs = a.nrhs;
  const CNodeDev nd = a.nodes[w.a];
  const double* row = a.B + nd.boff + (int64_t)w.row * nd.bld;
  const double* yp = a.y + (int64_t)nd.pos0 * nrhs;
  double* dst = a.u + (int64_t)a.order[nd.pos0 + w.row] * nrhs;
  if (ke - kb == 1) {
    const double s = warp_dot(row, yp, w.row, nd.p, nrhs, kb, lane) +
                     warp_dot_gather(row + nd.p, a.u, a.upd + nd.upd_off, nd.u, nrhs, kb, lane);
    if (lane == 0) dst[kb] = s;
    return;
  }
  for (int k0 = kb; k0 < ke; k0 += kNR) {
    const int nr = min(kNR, nrhs - k0);
    double s[kNR] = {0, 0, 0, 0, 0, 0, 0, 0};
    warp_dot_multi(row, yp, w.row, nd.p, nrhs, k0, nr, lane, s);
    warp_dot_gather_multi(row + nd.p, a.u, a.upd + nd.upd_off, nd.u, nrhs, k0, nr, lane, s);
    const double v = warp_sum8(s, lane);
    if ((lane & 3) == 0 && (lane >> 2) < nr) dst[k0 + (lane >> 2)] = v;
  }
}

// Row-blocked sweeps for several right-hand sides: a warp unit covers up to
// kRB consecutive rows of one node's matrix, so every operand value loaded
// feeds kRB rows. acc[q][k] += sum_j row_q[j] x[j, k0 + k] for j in [j0, j1);
// the operand is x[j * nrhs + ...] or, with idx, x[idx[j] * nrhs + ...].
constexpr int kRB = 4;
__device__ __forceinline__ void warp_rows_multi(const double* __restrict__ row, int ld, int nq, const double* x,
                                                const int32_t* __restrict__ idx, int j0, int j1, int nrhs, int k0,
                                                int nr, int lane, double (&s)[kRB][kNR]) {
  for (int j = j0 + lane; j < j1; j += 64) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int jj = j + 32 * t;
      const bool in = jj < j1;
      const int jc = in ? jj : j;
      double rv[kRB];
#pragma unroll
      for (int q = 0; q < kRB; ++q) rv[q] = (in && q < nq) ? __ldg(&row[(int64_t)q * ld + jc]) : 0.0;
      const int64_t xr = idx ? (int64_t)__ldg(&idx[jc - j0]) : (int64_t)jc;
      const double* xp = x + xr * nrhs + k0;
#pragma unroll
      for (int k = 0; k < kNR; ++k)
        if (k < nr) {
          const double xv = __ldcg(xp + k);
#pragma unroll
          for (int q = 0; q < kRB; ++q) s[q][k] = fma(rv[q], xv, s[q][k]);
        }
    }
  }
}

__device__ void forward_rows(const CoarseArgs& a, const CUnit& w, int lane, int kb, int ke) {
  // y[pos0 + i] = sum_{j <= i} L_PP^-1[i, j] r'[pos0 + j], i in [row, row + b)
  const int nrhs = a.nrhs, nq = w.b;
  const CNodeDev nd = a.nodes[w.a];
  const double* row = a.F + nd.foff + (int64_t)w.row * nd.fld;
  const double* x = a.rp + (int64_t)nd.pos0 * nrhs;
  for (int k0 = kb; k0 < ke; k0 += kNR) {
    const int nr = min(kNR, nrhs - k0);
    double s[kRB][kNR];
#pragma unroll
    for (int q = 0; q < kRB; ++q)
#pragma unroll
      for (int k = 0; k < kNR; ++k) s[q][k] = 0.0;
    warp_rows_multi(row, nd.fld, nq, x, nullptr, 0, w.row + nq, nrhs, k0, nr, lane, s);
#pragma unroll
    for (int q = 0; q < kRB; ++q) {
      const double v = warp_sum8(s[q], lane);
      if (q < nq && (lane & 3) == 0 && (lane >> 2) < nr)
        a.y[(int64_t)(nd.pos0 + w.row + q) * nrhs + k0 + (lane >> 2)] = v;
    }
  }
}

__device__ void backward_rows(const CoarseArgs& a, const CUnit& w, int lane, int kb, int ke) {
  // u[dof of pos0 + i] = sum_{j >= i} L_PP^-T[i, j] y[pos0 + j] - sum_b M[b, i] u[upd_b]
  const int nrhs = a.nrhs, nq = w.b;
  const CNodeDev nd = a.nodes[w.a];
  const double* row = a.B + nd.boff + (int64_t)w.row * nd.bld;
  const double* yp = a.y + (int64_t)nd.pos0 * nrhs;
  for (int k0 = kb; k0 < ke; k0 += kNR) {
    const int nr = min(kNR, nrhs - k0);
    double s[kRB][kNR];
#pragma unroll
    for (int q = 0; q < kRB; ++q)
#pragma unroll
      for (int k = 0; k < kNR; ++k) s[q][k] = 0.0;
    warp_rows_multi(row, nd.bld, nq, yp, nullptr, w.row, nd.p, nrhs, k0, nr, lane, s);
    warp_rows_multi(row + nd.p, nd.bld, nq, a.u, a.upd + nd.upd_off, 0, nd.u, nrhs, k0, nr, lane, s);
#pragma unroll
    for (int q = 0; q < kRB; ++q) {
      const double v = warp_sum8(s[q], lane);
      if (q < nq && (lane & 3) == 0 && (lane >> 2) < nr)
        a.u[(int64_t)a.order[nd.pos0 + w.row + q] * nrhs + k0 + (lane >> 2)] = v;
    }
  }
}

// RB = 1: one row per warp unit (one right-hand side, latency-bound);
// RB = kRB: row-blocked units (several right-hand sides).
template <int RB>
__global__ void __launch_bounds__(RB == 1 ? kThreads : kThreads / 2, 1) k_coarse_solve(CoarseArgs a) {
  const int L = a.levels;
  const int32_t* off_f = a.lvl;
  const int32_t* off_b = a.lvl + (L + 1);
  const int64_t n_c = a.lvl[2 * (L + 1)];
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  // a warp unit is (row unit, block of bw columns): the column blocks of one
  // unit run on different warps instead of one after the other. One-row
  // units take one column each (the single-column dot products); the
  // row-blocked units take kNR columns.
  const int bw = RB == 1 ? 1 : kNR;
  const int nrb = (a.nrhs + bw - 1) / bw;
  // r' = r_c in elimination order
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_c * a.nrhs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = i / a.nrhs;
    a.rp[i] = a.r[(int64_t)a.order[pos] * a.nrhs + (i - pos * a.nrhs)];
  }
  unsigned int epoch = 0;
  if (!grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
  for (int lv = 0; lv < L; ++lv) {
    for (int64_t t = (int64_t)off_f[lv] * nrb + gw; t < (int64_t)off_f[lv + 1] * nrb; t += nw) {
      const int64_t ui = t / nrb;
      const int kb = (int)(t - ui * nrb) * bw, ke = min(a.nrhs, kb + bw);
      const CUnit w = a.units[ui];
      if (RB > 1 && w.kind == 0)
        forward_rows(a, w, lane, kb, ke);
      else
        forward_unit(a, w, lane, kb, ke);
    }
    if (!grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
  }
  for (int lv = L - 1; lv >= 0; --lv) {
    for (int64_t t = (int64_t)off_b[lv] * nrb + gw; t < (int64_t)off_b[lv + 1] * nrb; t += nw) {
      const int64_t ui = t / nrb;
      const int kb = (int)(t - ui * nrb) * bw, ke = min(a.nrhs, kb + bw);
      if (RB > 1)
        backward_rows(a, a.units[ui], lane, kb, ke);
      else
        backward_unit(a, a.units[ui], lane, kb, ke);
    }
    if (lv > 0 && !grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
  }
}

// ---- gather form (one right-hand side) --------------------------------------------------
// One block per SM, at most 128 registers a thread: 512 threads when the
// sweeps run alone, 256 (half an SM's registers) when they overlap the
// interface operator, whose two streamed-GEMV blocks per SM then fit beside.
constexpr int kGThreadsWide = 512, kGThreadsNarrow = 256;
constexpr int kGU = 8;            // coefficients per lane per batch (256 per warp)
constexpr int kGBatch = 32 * kGU;
static_assert(kGBatch == kGatherBatch, "the warp assignment's cost unit is the kernel's batch");

struct GatherArgs {
  const CGUnit* units;
  const int32_t* wo;         // [2 L][warps + 1] descriptor offsets
  const double* C;
  const int32_t* I;
  const double* r;           // r_c (dof order)
  double* rp;                // r' (forward), then u (backward), elimination order
  double* y;                 // y (elimination order)
  double* u;                 // u_c (dof order)
  unsigned int* bar;
  int32_t* err;
  int levels, n_c;           // levels: forward-type phases (forward levels, then a dense top's product)
  unsigned int bar_extra;
  long long bar_cycles;
  int phases;                // all phases
};

// Coefficients and operand indices of one batch: elements base + lane + 32 i
// of a unit; past its end the index is -1 (the operand is not read).
__device__ __forceinline__ void gather_batch(const GatherArgs& a, int64_t off, int len, int base, int lane,
                                             double (&c)[kGU], int (&ix)[kGU]) {
#pragma unroll
  for (int i = 0; i < kGU; ++i) {
    const int j = base + lane + 32 * i;
    const bool in = j < len;
    c[i] = in ? __ldg(a.C + off + j) : 0.0;
    ix[i] = in ? __ldg(a.I + off + j) : -1;
  }
}

// Lane l holds the descriptor of the warp's unit m0 + l of a phase.
__device__ __forceinline__ CGUnit gather_desc(const GatherArgs& a, int beg, int cnt, int m0, int lane) {
  CGUnit d{0, 0, 0, 0, 0};
  if (m0 + lane < cnt) d = a.units[beg + m0 + lane];
  return d;
}

__device__ __forceinline__ double gather_x(const double* A, const double* B, int n_c, int ix) {
  return __ldcg(ix < n_c ? A + ix : B + (ix - n_c));
}

template <int NT>
__global__ void __launch_bounds__(NT, kGThreadsWide / NT) k_coarse_sweeps(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (NT / 32);
  const int gw = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  const int P = a.phases;
  unsigned int epoch = 0;
  int beg = a.wo[gw], cnt = a.wo[gw + 1] - beg;
  CGUnit dl = gather_desc(a, beg, cnt, 0, lane);
  // nc / nix: the batch to be used next, loaded ahead (pre)
  double nc[kGU];
  int nix[kGU];
  bool pre = false;
  if (cnt > 0) {
    gather_batch(a, __shfl_sync(0xffffffffu, dl.off, 0), __shfl_sync(0xffffffffu, dl.len, 0), 0, lane, nc, nix);
    pre = true;
  }
  for (int ph = 0; ph < P; ++ph) {
    int nbeg = 0, ncnt = 0;
    CGUnit ndl{0, 0, 0, 0, 0};
    if (ph + 1 < P) {
      const int32_t* w = a.wo + (int64_t)(ph + 1) * (nw + 1) + gw;
      nbeg = w[0];
      ncnt = w[1] - nbeg;
      ndl = gather_desc(a, nbeg, ncnt, 0, lane);
    }
    const bool fwd = ph < a.levels;
    const double* XA = fwd ? a.rp : a.y;
    const double* XB = fwd ? a.r : a.rp;
    for (int m = 0; m < cnt; ++m) {
      if (m > 0 && (m & 31) == 0) dl = gather_desc(a, beg, cnt, m, lane);
      const int sl = m & 31;
      const int64_t off = __shfl_sync(0xffffffffu, dl.off, sl);
      const int len = __shfl_sync(0xffffffffu, dl.len, sl);
      const int dst = __shfl_sync(0xffffffffu, dl.dst, sl);
      const int aux = __shfl_sync(0xffffffffu, dl.aux, sl);
      if (!pre) gather_batch(a, off, len, 0, lane, nc, nix);
      double s = 0.0, x0 = 0.0;
      for (int base = 0; base < len; base += kGBatch) {
        double c[kGU], xv[kGU];
        int ix[kGU];
#pragma unroll
        for (int i = 0; i < kGU; ++i) {
          c[i] = nc[i];
          ix[i] = nix[i];
        }
#pragma unroll
        for (int i = 0; i < kGU; ++i) xv[i] = ix[i] >= 0 ? gather_x(XA, XB, a.n_c, ix[i]) : 0.0;
        if (base == 0 && fwd && aux >= 0) x0 = gather_x(XA, XB, a.n_c, aux);
        // the next batch: of this unit, else the first of the next unit
        // (this phase or the next one)
        pre = true;
        if (base + kGBatch < len) {
          gather_batch(a, off, len, base + kGBatch, lane, nc, nix);
        } else if (m + 1 < cnt) {
          const int s2 = (m + 1) & 31;
          if (s2 != 0)
            gather_batch(a, __shfl_sync(0xffffffffu, dl.off, s2), __shfl_sync(0xffffffffu, dl.len, s2), 0, lane,
                         nc, nix);
          else
            pre = false;
        } else if (ncnt > 0) {
          gather_batch(a, __shfl_sync(0xffffffffu, ndl.off, 0), __shfl_sync(0xffffffffu, ndl.len, 0), 0, lane, nc,
                       nix);
        } else {
          pre = false;
        }
#pragma unroll
        for (int i = 0; i < kGU; ++i) s = fma(c[i], xv[i], s);
      }
      s = warp_sum(s);
      if (lane == 0) {
        if (!fwd) {
          a.rp[dst] = s;
          a.u[aux] = s;
        } else if (aux < 0) {
          a.y[dst] = s;
        } else {
          a.rp[dst] = x0 - s;
        }
      }
    }
    if (cnt == 0) {
      pre = false;
      if (ncnt > 0) {
        gather_batch(a, __shfl_sync(0xffffffffu, ndl.off, 0), __shfl_sync(0xffffffffu, ndl.len, 0), 0, lane, nc,
                     nix);
        pre = true;
      }
    }
    if (ph + 1 < P && !grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
    beg = nbeg;
    cnt = ncnt;
    dl = ndl;
  }
}


// ---- per-level form (one right-hand side, large factors) --------------------------------
// One launch per phase of the gather form (the launch boundary replaces the
// grid barrier, and the grid is not limited to one resident block per SM).
// A phase's units, longest first, are split into classes by length; a unit
// of class c is processed by a group of G = 32, 16, 8, 4, 2 or 1 lanes, so
// the many short rows of the lower levels keep every lane busy: each lane
// strides over the unit's coefficients four at a time (their operand loads
// in flight together), the group's partial sums are combined by shuffles
// within the group, and its first lane stores the result. Values of other
// phases are read with plain loads (written by earlier launches);
// coefficients and indices through the read-only path.
// TC: the coefficients' type. double: float64 products and sums; float
// (the mixed forms of the sparse local solver): float32 coefficients,
// products and sums, which moves the products from the float64 pipe (a few
// per SM and cycle on this GPU) to the float32 pipe and reads 8 bytes per
// coefficient instead of 12. The operands are float32 copies of r', y and r
// (xa32, xb32), each value rounded once where it is written (rp32, y32; r
// by k_round_f32 before the forward sweep), because a float64 -> float32
// conversion also runs on the float64 pipe and, done per coefficient, kept
// that pipe as busy as the products did. The results are the same as with
// the rounding at each read. The float64 vectors are still written: the
// receiving units' r'_U - s and the result u stay in float64.
template <typename TC>
struct LevelArgs {
  const CGUnit* units;       // the phase's descriptors
  const TC* C;
  const int32_t* I;
  const double* xa;          // operand vector for indices < n (forward: r', backward: y)
  const double* xb;          // operand vector for indices n + i (forward: r, backward: u by position)
  double* rp;                // r' (forward, receiving units) / u by position (backward)
  double* y;                 // y (forward rows)
  double* u;                 // u by dof (backward)
  int n, fwd;
  int32_t cb[kLevelClasses + 1], bb[kLevelClasses + 1];
  const float* xa32 = nullptr;   // TC = float: float32 copies of xa and xb
  const float* xb32 = nullptr;
  float* rp32 = nullptr;         // TC = float: float32 copies of rp and y, written with them
  float* y32 = nullptr;
};

// f[i] = r[i] rounded to float32 (the forward sweep's operand r in the
// float32 form of the per-level sweeps)
__global__ void k_round_f32(const double* __restrict__ r, float* __restrict__ f, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) f[i] = (float)r[i];
}

template <typename TC, int G, int c>
__device__ __forceinline__ void level_group(const LevelArgs<TC>& a, int b) {
  const int grp = (int)threadIdx.x / G, gl = (int)threadIdx.x % G;
  const int k = a.cb[c] + (b - a.bb[c]) * (kLevelThreads / G) + grp;
  const bool valid = k < a.cb[c + 1];
  CGUnit d{0, 0, 0, -1, 0};
  if (valid) d = a.units[k];
  const TC* C = a.C + d.off;
  const int32_t* I = a.I + d.off;
  constexpr bool kF32 = std::is_same<TC, float>::value;
  auto X = [&](int ix) { return ix < a.n ? a.xa[ix] : a.xb[ix - a.n]; };
  // operand of a coefficient in the coefficients' type
  auto XO = [&](int ix) -> TC {
    if constexpr (kF32)
      return ix < a.n ? a.xa32[ix] : a.xb32[ix - a.n];
    else
      return X(ix);
  };
  TC s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int j = gl; j < d.len; j += 4 * G) {
    const bool b1 = j + G < d.len, b2 = j + 2 * G < d.len, b3 = j + 3 * G < d.len;
    const TC c0 = __ldg(C + j);
    const TC c1 = b1 ? __ldg(C + j + G) : TC(0);
    const TC c2 = b2 ? __ldg(C + j + 2 * G) : TC(0);
    const TC c3 = b3 ? __ldg(C + j + 3 * G) : TC(0);
    const int i0 = __ldg(I + j);
    const int i1 = b1 ? __ldg(I + j + G) : i0;
    const int i2 = b2 ? __ldg(I + j + 2 * G) : i0;
    const int i3 = b3 ? __ldg(I + j + 3 * G) : i0;
    const TC x0 = XO(i0), x1 = XO(i1), x2 = XO(i2), x3 = XO(i3);
    s0 = fma(c0, x0, s0);
    s1 = fma(c1, x1, s1);
    s2 = fma(c2, x2, s2);
    s3 = fma(c3, x3, s3);
  }
  TC s = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (!valid || gl != 0) return;
  if (!a.fwd) {
    a.rp[d.dst] = (double)s;
    a.u[d.aux] = (double)s;
    if constexpr (kF32) a.rp32[d.dst] = (float)s;
  } else if (d.aux < 0) {
    a.y[d.dst] = (double)s;
    if constexpr (kF32) a.y32[d.dst] = (float)s;
  } else {
    const double v = X(d.aux) - (double)s;
    a.rp[d.dst] = v;
    if constexpr (kF32) a.rp32[d.dst] = (float)v;
  }
}

template <typename TC>
__global__ void __launch_bounds__(kLevelThreads) k_level_sweep(LevelArgs<TC> a) {
  const int b = blockIdx.x;
  int c = 0;   // the block's class (the block ranges ascend with the class)
#pragma unroll
  for (int q = 1; q < kLevelClasses; ++q) c += b >= a.bb[q];
  switch (c) {
    case 0: level_group<TC, 32, 0>(a, b); break;
    case 1: level_group<TC, 16, 1>(a, b); break;
    case 2: level_group<TC, 8, 2>(a, b); break;
    case 3: level_group<TC, 4, 3>(a, b); break;
    case 4: level_group<TC, 2, 4>(a, b); break;
    default: level_group<TC, 1, 5>(a, b); break;
  }
}

// ---- block form (one right-hand side, large factors) --------------------------------------
// One launch per phase; one block per work item (a chunk of rows of one
// supernode). The block assembles the node's front vector in shared memory
// (forward: r at the pivots plus the children's contribution vectors,
// children one after another so the sums have a fixed order; backward: y at
// the pivots and u at the update set's positions), then groups of G lanes
// take one row each: the row's coefficients are read contiguously (four per
// lane in flight), multiplied with the front from shared memory and summed
// by shuffles within the group.
constexpr int kBlockThreads = 256;

struct BlockArgs {
  const SNode* nodes;
  const int32_t* kids;
  const int32_t* cmap;
  const int32_t* upd;
  const BlockItem* items;    // this phase's items
  const double* F;
  const double* B;
  const double* r;           // right-hand side at the pivots (positions): r, or r' after gather-form levels
  double* y;                 // forward result (positions)
  double* u;                 // solution (positions)
  double* cbuf;              // contribution vectors
  int kmin;                  // children below this height ran the gather form (their contributions are in r')
};

// sum over j in [j0, j1) of m[j] v[j] by a group of G lanes (lane gl), the
// total on every lane of the group
template <int G>
__device__ __forceinline__ double group_dot(const double* __restrict__ m, const double* v, int j0, int j1, int gl) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int j = j0 + gl; j < j1; j += 4 * G) {
    const bool b1 = j + G < j1, b2 = j + 2 * G < j1, b3 = j + 3 * G < j1;
    const double m0 = __ldg(m + j);
    const double m1 = b1 ? __ldg(m + j + G) : 0.0;
    const double m2 = b2 ? __ldg(m + j + 2 * G) : 0.0;
    const double m3 = b3 ? __ldg(m + j + 3 * G) : 0.0;
    s0 = fma(m0, v[j], s0);
    s1 = fma(m1, b1 ? v[j + G] : 0.0, s1);
    s2 = fma(m2, b2 ? v[j + 2 * G] : 0.0, s2);
    s3 = fma(m3, b3 ? v[j + 3 * G] : 0.0, s3);
  }
  double s = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Rows [row0, row0 + nrows) of node d by groups of G lanes: thread t of the
// cooperating threads (T of them: a block, or a warp for a small node) is
// lane t % G of group t / G.
template <int G, int T>
__device__ __forceinline__ void block_fwd_rows(const BlockArgs& a, int row0, int nrows, const SNode& d,
                                               const double* f, int t) {
  const int grp = t / G, gl = t % G;
  const int end = row0 + nrows;
  for (int base = row0; base < end; base += T / G) {
    const int row = base + grp;
    const bool valid = row < end;
    const int len = !valid ? 0 : row < d.p ? row + 1 : d.p;
    const double s = group_dot<G>(a.F + d.foff + (int64_t)(valid ? row : 0) * d.fld, f, 0, len, gl);
    if (valid && gl == 0) {
      if (row < d.p)
        a.y[d.pos0 + row] = s;
      else
        a.cbuf[d.cbase + row - d.p] = f[row] - s;
    }
  }
}

template <int G, int T>
__device__ __forceinline__ void block_bwd_rows(const BlockArgs& a, int row0, int nrows, const SNode& d,
                                               const double* v, int t) {
  const int grp = t / G, gl = t % G;
  const int end = row0 + nrows, f = d.p + d.u;
  for (int base = row0; base < end; base += T / G) {
    const int row = base + grp;
    const bool valid = row < end;
    const double s = group_dot<G>(a.B + d.boff + (int64_t)(valid ? row : 0) * d.bld, v, valid ? row : f, f, gl);
    if (valid && gl == 0) a.u[d.pos0 + row] = s;
  }
}

template <int T>
__device__ __forceinline__ void fwd_rows(const BlockArgs& a, const BlockItem& it, const SNode& d, const double* f,
                                         int t) {
  switch (it.g) {
    case 32: block_fwd_rows<32, T>(a, it.row0, it.nrows, d, f, t); break;
    case 16: block_fwd_rows<16, T>(a, it.row0, it.nrows, d, f, t); break;
    case 8: block_fwd_rows<8, T>(a, it.row0, it.nrows, d, f, t); break;
    default: block_fwd_rows<4, T>(a, it.row0, it.nrows, d, f, t); break;
  }
}
template <int T>
__device__ __forceinline__ void bwd_rows(const BlockArgs& a, const BlockItem& it, const SNode& d, const double* v,
                                         int t) {
  switch (it.g) {
    case 32: block_bwd_rows<32, T>(a, it.row0, it.nrows, d, v, t); break;
    case 16: block_bwd_rows<16, T>(a, it.row0, it.nrows, d, v, t); break;
    case 8: block_bwd_rows<8, T>(a, it.row0, it.nrows, d, v, t); break;
    default: block_bwd_rows<4, T>(a, it.row0, it.nrows, d, v, t); break;
  }
}

// Blocks [0, nbig): one chunk of a large node each (the front assembled by
// the whole block); the later blocks: kBlockThreads / 32 small nodes each,
// one per warp (its front in the warp's slice of kSmallFront values).
__global__ void __launch_bounds__(kBlockThreads) k_block_fwd(BlockArgs a, int nbig, int nitems) {
  extern __shared__ double smem[];
  if ((int)blockIdx.x < nbig) {
    const BlockItem it = a.items[blockIdx.x];
    const SNode d = a.nodes[it.node];
    const int f = d.p + d.u;
    for (int i = threadIdx.x; i < f; i += kBlockThreads) smem[i] = i < d.p ? a.r[d.pos0 + i] : 0.0;
    __syncthreads();
    for (int q = 0; q < d.nkid; ++q) {
      const SNode k = a.nodes[a.kids[d.kid0 + q]];
      if (k.height < a.kmin) continue;   // uniform across the block
      for (int i = threadIdx.x; i < k.u; i += kBlockThreads) smem[a.cmap[k.cmap0 + i]] += a.cbuf[k.cbase + i];
      __syncthreads();
    }
    fwd_rows<kBlockThreads>(a, it, d, smem, threadIdx.x);
    return;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = nbig + ((int)blockIdx.x - nbig) * (kBlockThreads / 32) + w;
  if (k >= nitems) return;   // the whole warp (no block-wide barrier below)
  double* f = smem + w * kSmallFront;
  const BlockItem it = a.items[k];
  const SNode d = a.nodes[it.node];
  const int fs = d.p + d.u;
  for (int i = lane; i < fs; i += 32) f[i] = i < d.p ? a.r[d.pos0 + i] : 0.0;
  __syncwarp();
  for (int q = 0; q < d.nkid; ++q) {
    const SNode kd = a.nodes[a.kids[d.kid0 + q]];
    if (kd.height < a.kmin) continue;
    for (int i = lane; i < kd.u; i += 32) f[a.cmap[kd.cmap0 + i]] += a.cbuf[kd.cbase + i];
    __syncwarp();
  }
  fwd_rows<32>(a, it, d, f, lane);
}

__global__ void __launch_bounds__(kBlockThreads) k_block_bwd(BlockArgs a, int nbig, int nitems) {
  extern __shared__ double smem[];
  if ((int)blockIdx.x < nbig) {
    const BlockItem it = a.items[blockIdx.x];
    const SNode d = a.nodes[it.node];
    const int f = d.p + d.u;
    for (int i = threadIdx.x; i < f; i += kBlockThreads)
      smem[i] = i < d.p ? a.y[d.pos0 + i] : a.u[a.upd[d.upd_off + i - d.p]];
    __syncthreads();
    bwd_rows<kBlockThreads>(a, it, d, smem, threadIdx.x);
    return;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = nbig + ((int)blockIdx.x - nbig) * (kBlockThreads / 32) + w;
  if (k >= nitems) return;
  double* v = smem + w * kSmallFront;
  const BlockItem it = a.items[k];
  const SNode d = a.nodes[it.node];
  const int fs = d.p + d.u;
  for (int i = lane; i < fs; i += 32) v[i] = i < d.p ? a.y[d.pos0 + i] : a.u[a.upd[d.upd_off + i - d.p]];
  __syncwarp();
  bwd_rows<32>(a, it, d, v, lane);
}

// ---- inexact coarse solve: plain CG on A_c (all columns in lockstep) ---------------------
//
// One cooperative persistent launch per coarse solve. Rows of A_c (CSR, glob
// order) are dealt over the grid's threads, one (row, column) pair per thread
// step; every reduction is a per-block partial in a fixed slot, summed in
// block order by every block after a grid barrier, so all blocks take the
// same decisions (step lengths, stop test, loop count) and the result does
// not depend on timing. Three barriers per iteration: after q = A_c p with
// p.q, after the updates of u and r with r.r, and after the update of p.
constexpr int kCgThreadsWide = 512, kCgThreadsNarrow = 256;
constexpr int kCgMaxRhs = 64;

struct CgArgs {
  const int32_t* ptr;        // [n_c + 1]
  const int32_t* col;
  const double* val;
  const double* rc;          // r_c, n_c x nrhs (dof-major, column fastest)
  double* u;                 // u_c
  double* r;                 // residual
  double* p;                 // search direction
  double* q;                 // A_c p
  double* part;              // [grid][2][nrhs] block partial sums
  int32_t* iters;            // [nrhs] iterations of this solve
  unsigned int* bar;
  int32_t* err;
  int n_c, nrhs, maxit;
  double rtol;
  unsigned int bar_extra;
  long long bar_cycles;
};

// The block's sums of s per column (thread t holds column t % nrhs) into
// part[blockIdx.x][slot][k], in a fixed order.
__device__ void cg_block_partial(double s, const CgArgs& a, int slot, double* red) {
  const int t = threadIdx.x, per = blockDim.x / a.nrhs;
  red[t] = t < per * a.nrhs ? s : 0.0;
  __syncthreads();
  if (t < a.nrhs) {
    double v = 0.0;
    for (int j = 0; j < per; ++j) v += red[j * a.nrhs + t];
    a.part[((int64_t)blockIdx.x * 2 + slot) * a.nrhs + t] = v;
  }
  __syncthreads();
}
// Totals of a slot over all blocks, in block order, into tot[k] (shared).
__device__ void cg_total(const CgArgs& a, int slot, double* tot) {
  const int t = threadIdx.x;
  if (t < a.nrhs) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(&a.part[((int64_t)b * 2 + slot) * a.nrhs + t]);
    tot[t] = v;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCgThreadsWide) k_coarse_cg(CgArgs a) {
  __shared__ double red[kCgThreadsWide];
  __shared__ double tot[kCgMaxRhs], rho[kCgMaxRhs], tol2[kCgMaxRhs], alpha[kCgMaxRhs], beta[kCgMaxRhs];
  __shared__ int active[kCgMaxRhs], n_active;
  const int nr = a.nrhs, per = blockDim.x / nr;
  const int sub = threadIdx.x / nr, k = threadIdx.x - sub * nr;
  const bool live = threadIdx.x < per * nr;
  const int64_t stride = (int64_t)gridDim.x * per;
  unsigned int epoch = 0;
  // u = 0, r = p = r_c, and r.r
  double s = 0.0;
  if (live)
    for (int64_t i = blockIdx.x * (int64_t)per + sub; i < a.n_c; i += stride) {
      const int64_t e = i * nr + k;
      const double v = a.rc[e];
      a.u[e] = 0.0;
      a.r[e] = v;
      a.p[e] = v;
      s = fma(v, v, s);
    }
  cg_block_partial(s, a, 0, red);
  if (!grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
  cg_total(a, 0, tot);
  if (threadIdx.x < nr) {
    const int t = threadIdx.x;
    rho[t] = tot[t];
    tol2[t] = a.rtol * a.rtol * tot[t];
    active[t] = tot[t] > tol2[t] ? 1 : 0;   // a zero column takes no iteration
    if (blockIdx.x == 0) a.iters[t] = 0;
  }
  if (threadIdx.x == 0) n_active = 0;
  __syncthreads();
  if (threadIdx.x < nr && active[threadIdx.x]) atomicAdd(&n_active, 1);
  __syncthreads();
  for (int it = 0; it < a.maxit && n_active > 0; ++it) {
    // q = A_c p and p.q
    s = 0.0;
    if (live)
      for (int64_t i = blockIdx.x * (int64_t)per + sub; i < a.n_c; i += stride) {
        double acc = 0.0;
        const int j1 = a.ptr[i + 1];
        for (int j = a.ptr[i]; j < j1; ++j) acc = fma(a.val[j], __ldcg(&a.p[(int64_t)a.col[j] * nr + k]), acc);
        a.q[i * nr + k] = acc;
        s = fma(__ldcg(&a.p[i * nr + k]), acc, s);
      }
    cg_block_partial(s, a, 1, red);
    if (!grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
    cg_total(a, 1, tot);
    if (threadIdx.x < nr) {
      const int t = threadIdx.x;
      alpha[t] = active[t] && tot[t] > 0.0 ? rho[t] / tot[t] : 0.0;
    }
    __syncthreads();
    // u += alpha p, r -= alpha q, and r.r
    s = 0.0;
    if (live) {
      const double al = alpha[k];
      for (int64_t i = blockIdx.x * (int64_t)per + sub; i < a.n_c; i += stride) {
        const int64_t e = i * nr + k;
        const double pe = __ldcg(&a.p[e]);
        a.u[e] = fma(al, pe, a.u[e]);
        const double re = fma(-al, a.q[e], a.r[e]);
        a.r[e] = re;
        s = fma(re, re, s);
      }
    }
    cg_block_partial(s, a, 0, red);
    if (!grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
    cg_total(a, 0, tot);
    if (threadIdx.x == 0) n_active = 0;
    __syncthreads();
    if (threadIdx.x < nr) {
      const int t = threadIdx.x;
      beta[t] = 0.0;
      if (active[t]) {
        if (blockIdx.x == 0) a.iters[t] = it + 1;
        beta[t] = rho[t] > 0.0 ? tot[t] / rho[t] : 0.0;
        rho[t] = tot[t];
        if (!(tot[t] > tol2[t])) active[t] = 0;   // converged (or not finite)
        else atomicAdd(&n_active, 1);
      }
    }
    __syncthreads();
    // p = r + beta p (the columns that go on)
    if (live && active[k]) {
      const double be = beta[k];
      for (int64_t i = blockIdx.x * (int64_t)per + sub; i < a.n_c; i += stride) {
        const int64_t e = i * nr + k;
        a.p[e] = fma(be, a.p[e], a.r[e]);
      }
    }
    if (!grid_sync(a.bar, a.err, epoch, a.bar_extra, a.bar_cycles)) return;
  }
}

template <typename T>
cudaError_t up(bddc_handle_s* h, T** dst, const std::vector<T>& v) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocations.push_back(p);
  *dst = static_cast<T*>(p);
  if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace


namespace {

cudaError_t build_gather(bddc_handle_s* h, const CoarseFactor& cf, SweepSet& S, int blocks, bool level_form,
                         bool coef32) {
  GatherLayout g;
  const int nb[2] = {blocks, blocks}, wpb[2] = {kGThreadsWide / 32, kGThreadsNarrow / 32};
  gather_layout(cf, level_form ? 0 : 2, nb, wpb, g);
  S.g_entries = (int64_t)g.C.size();
  S.g_blocks = blocks;
  S.g_fwd = g.fwd_phases;
  S.g_phases = g.phases;
  const int L = cf.n_levels;
  S.gbytes_h.assign(L, 0);
  if (level_form && g.phases == 2 * L)
    for (int ph = 0; ph < 2 * L; ++ph) {
      int64_t len = 0;
      for (int64_t k = g.seq_off[ph]; k < g.seq_off[ph + 1]; ++k) len += g.seq[k].len;
      S.gbytes_h[ph < L ? ph : 2 * L - 1 - ph] += 12 * len;
    }
  cudaError_t e;
  if (coef32) {
    // the per-level form only (the cooperative kernel reads float64)
    std::vector<float> c32(g.C.begin(), g.C.end());
    std::vector<double>().swap(g.C);
    if ((e = up(h, &S.gC32, c32)) != cudaSuccess) return e;
    // float32 copies of the operand vectors r', y and r, so that the
    // per-coefficient operand loads need no float64 -> float32 conversion
    if ((e = up(h, &S.x32, std::vector<float>(3 * (size_t)cf.n, 0.0f))) != cudaSuccess) return e;
  } else {
    if ((e = up(h, &S.gC, g.C)) != cudaSuccess) return e;
    std::vector<double>().swap(g.C);
  }
  if ((e = up(h, &S.gI, g.I)) != cudaSuccess) return e;
  std::vector<int32_t>().swap(g.I);
  // the per-level form always (for the cooperative form it is the
  // alternative the autotuner measures)
  level_phases(g, S.lv);
  if ((e = up(h, &S.seq, g.seq)) != cudaSuccess) return e;
  S.use_level = level_form;
  if (level_form) return cudaSuccess;
  for (int sh = 0; sh < 2; ++sh) {
    if ((e = up(h, &S.gU[sh], g.units[sh])) != cudaSuccess) return e;
    if ((e = up(h, &S.gwo[sh], g.wo[sh])) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t build_coarse_cg_device(bddc_handle_s* h) {
  cudaError_t e;
  if ((e = up(h, &h->d_cbar, std::vector<unsigned int>(2, 0u))) != cudaSuccess) return e;
  int dev = 0, coop = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  // one block per SM must be resident, in both shapes (cooperative grid)
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_cg, kCgThreadsWide, 0)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  return cudaSuccess;
}

cudaError_t build_sweeps(bddc_handle_s* h, const CoarseFactor& cf, SweepSet& S, bool multi, int blocks_req,
                         int form, bool coef32) {
  if (coef32 && form == kSweepCoop) return cudaErrorInvalidValue;
  const int L = cf.n_levels;
  S.levels = L;
  S.n = cf.n;
  S.multi = multi;
  if (cf.n == 0) return cudaSuccess;
  const int nn = (int)cf.nodes.size();
  std::vector<CNodeDev> nodes(nn);
  std::vector<int32_t> upd;
  int64_t fcur = 0, bcur = 0, ucur = 0;
  for (int t = 0; t < nn; ++t) {
    const CoarseNode& T = cf.nodes[t];
    CNodeDev d{};
    d.p = T.p;
    d.u = T.u;
    d.pos0 = T.last - T.p + 1;
    d.upd_off = (int32_t)upd.size();
    d.fld = std::max(T.p, 1);
    d.bld = std::max(T.p + T.u, 1);
    fcur = (fcur + 31) / 32 * 32;
    d.foff = fcur;
    fcur += (int64_t)(T.p + T.u) * d.fld;
    bcur = (bcur + 31) / 32 * 32;
    d.boff = bcur;
    bcur += (int64_t)T.p * d.bld;
    if (multi) upd.insert(upd.end(), T.upd.begin(), T.upd.end());
    ucur += T.u;
    nodes[t] = d;
  }
  S.nnz = fcur + bcur;
  S.update_total = ucur;
  cudaError_t e;
  if (S.bar == nullptr && (e = up(h, &S.bar, std::vector<unsigned int>(2, 0u))) != cudaSuccess) return e;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  // cooperative grids: every block resident at once, in every shape
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_sweeps<kGThreadsWide>, kGThreadsWide,
                                                         0)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_sweeps<kGThreadsNarrow>,
                                                         kGThreadsNarrow, 0)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  // one-column form: the block form where every front fits in shared
  // memory, else the per-level gather form
  BlockLayout bl;
  bool block = form == kSweepBlock && !coef32;
  if (block) {
    block_layout(cf, kBlockTarget, bl);
    block = bl.max_front <= kBlockMaxFront;
    for (int t = 0; t < nn && block; ++t)
      if (bl.nodes[t].foff != nodes[t].foff || bl.nodes[t].boff != nodes[t].boff) return cudaErrorInvalidValue;
  }
  // the gather form (the block form keeps its per-level launches for the
  // low levels, whose nodes are too small for a block of their own)
  if ((e = build_gather(h, cf, S, blocks_req > 0 ? std::min(blocks_req, sms) : sms, form != kSweepCoop, coef32)) !=
      cudaSuccess)
    return e;
  S.read_1col = S.g_entries * (coef32 ? 8 : 12);
  if (block) {
    S.block_form = true;
    S.bitem_off = bl.item_off;
    S.bn_big = bl.n_big;
    S.bphase_front.assign(bl.item_off.size() - 1, 0);
    int64_t entries = 0;
    for (size_t ph = 0; ph + 1 < bl.item_off.size(); ++ph)
      for (int64_t k = bl.item_off[ph]; k < bl.item_off[ph + 1]; ++k) {
        const SNode& d = bl.nodes[bl.items[k].node];
        if (k < bl.item_off[ph] + bl.n_big[ph]) S.bphase_front[ph] = std::max(S.bphase_front[ph], d.p + d.u);
      }
    // default split: every level in the gather form (measured fastest on the
    // 2D workloads of 10^4 and 7.8 10^4 dofs per subdomain, each level
    // against the block form); the autotuner tries every split
    S.block_min_height = L;
    // bytes of one one-column solve per height: the block form reads the
    // lower part of F and the upper part of B once each, the gather form its
    // coefficients and indices
    S.bbytes_h.assign(L, 0);
    for (const SNode& d : bl.nodes) {
      const int64_t ent = (int64_t)d.p * (d.p + 1) / 2 + (int64_t)d.u * d.p;
      S.bbytes_h[d.height] += 2 * 8 * ent;
      entries += ent;
    }
    if ((e = up(h, &S.bnodes, bl.nodes)) != cudaSuccess) return e;
    if ((e = up(h, &S.bkids, bl.kids)) != cudaSuccess) return e;
    if ((e = up(h, &S.bcmap, bl.cmap)) != cudaSuccess) return e;
    if ((e = up(h, &S.bupd, bl.upd)) != cudaSuccess) return e;
    if ((e = up(h, &S.bitems, bl.items)) != cudaSuccess) return e;
    if ((e = up(h, &S.cbuf, std::vector<double>((size_t)std::max<int64_t>(bl.cbuf, 1), 0.0))) != cudaSuccess)
      return e;
    const int smem = bl.max_front * (int)sizeof(double);
    if (smem > 48 * 1024) {
      if ((e = cudaFuncSetAttribute(k_block_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(k_block_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return e;
    }
  }
  if (!multi && !block) return cudaSuccess;
  std::vector<double> F, B;
  if (block) {
    // the block layout's node matrices: the same offsets (same order and alignment)
    F.swap(bl.F);
    B.swap(bl.B);
  } else {
    F.assign((size_t)std::max<int64_t>(fcur, 1), 0.0);
    B.assign((size_t)std::max<int64_t>(bcur, 1), 0.0);
    for (int t = 0; t < nn; ++t) {
      const CoarseNode& T = cf.nodes[t];
      const int f = T.p + T.u;
      for (int r = 0; r < f; ++r)
        std::memcpy(&F[nodes[t].foff + (int64_t)r * nodes[t].fld], &T.Fm[(size_t)r * T.p], sizeof(double) * T.p);
      for (int r = 0; r < T.p; ++r)
        std::memcpy(&B[nodes[t].boff + (int64_t)r * nodes[t].bld], &T.Bm[(size_t)r * f], sizeof(double) * f);
    }
  }
  std::vector<int32_t> pos(cf.n);
  for (int64_t i = 0; i < cf.n; ++i) pos[cf.order[i]] = (int32_t)i;
  // warp units: forward levels (L_PP^-1 rows, then one unit per receiving
  // position with its (node, M row) pairs in node order), then backward
  // levels; rows of kinds 0 and 2 in blocks of rb (1, or kRB for the
  // multi-RHS sweeps). The contribution list is the same for both blockings.
  std::vector<CContrib> list;
  std::vector<std::vector<int32_t>> contrib(cf.n);
  std::vector<int32_t> touched;
  auto make_units = [&](int rb, std::vector<CUnit>& units, std::vector<int32_t>& lvl, bool fill_list) {
    lvl.assign(2 * (L + 1) + 1, 0);
    int32_t lcur = 0;
    for (int lv = 0; lv < L; ++lv) {
      lvl[lv] = (int)units.size();
      touched.clear();
      for (int t = 0; t < nn; ++t) {
        const CoarseNode& T = cf.nodes[t];
        if (T.height != lv || T.p == 0) continue;
        for (int i = 0; i < T.p; i += rb) units.push_back(CUnit{0, t, i, std::min(rb, T.p - i), 0});
        for (int b = 0; b < T.u; ++b) {
          const int32_t w = pos[T.upd[b]];
          if (contrib[w].empty()) touched.push_back(w);
          contrib[w].push_back(t);
          contrib[w].push_back(b);
        }
      }
      std::sort(touched.begin(), touched.end());
      for (int32_t w : touched) {
        const int32_t b0 = lcur;
        for (size_t q = 0; q < contrib[w].size(); q += 2) {
          const CNodeDev& nd = nodes[contrib[w][q]];
          if (fill_list) list.push_back(CContrib{nd.foff + (int64_t)(nd.p + contrib[w][q + 1]) * nd.fld, nd.pos0, nd.p, 0});
          ++lcur;
        }
        units.push_back(CUnit{1, w, 0, b0, lcur});
        contrib[w].clear();
      }
    }
    lvl[L] = (int)units.size();
    for (int lv = 0; lv < L; ++lv) {
      lvl[(L + 1) + lv] = (int)units.size();
      for (int t = 0; t < nn; ++t) {
        const CoarseNode& T = cf.nodes[t];
        if (T.height != lv || T.p == 0) continue;
        for (int i = 0; i < T.p; i += rb) units.push_back(CUnit{2, t, i, std::min(rb, T.p - i), 0});
      }
    }
    lvl[(L + 1) + L] = (int)units.size();
    lvl[2 * (L + 1)] = (int32_t)cf.n;
  };
  std::vector<CUnit> units, units4;
  std::vector<int32_t> lvl, lvl4;
  make_units(1, units, lvl, true);
  make_units(kRB, units4, lvl4, false);
  if ((e = up(h, &S.F, F)) != cudaSuccess) return e;
  std::vector<double>().swap(F);
  if ((e = up(h, &S.B, B)) != cudaSuccess) return e;
  std::vector<double>().swap(B);
  if (!multi) return cudaSuccess;
  if ((e = up(h, &S.nodes, nodes)) != cudaSuccess) return e;
  if ((e = up(h, &S.units, units)) != cudaSuccess) return e;
  if ((e = up(h, &S.units4, units4)) != cudaSuccess) return e;
  if ((e = up(h, &S.lvl4, lvl4)) != cudaSuccess) return e;
  if ((e = up(h, &S.list, list)) != cudaSuccess) return e;
  if ((e = up(h, &S.upd, upd)) != cudaSuccess) return e;
  if ((e = up(h, &S.order, cf.order)) != cudaSuccess) return e;
  if ((e = up(h, &S.lvl, lvl)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_solve<1>, kThreads, 0)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  S.grid = sms * std::min(per_sm, 2);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_solve<kRB>, kThreads / 2, 0)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  S.grid4 = sms * std::min(per_sm, 2);
  return cudaSuccess;
}

cudaError_t build_coarse_device(bddc_handle_s* h, const CoarseFactor& cf) {
  int dev = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  cudaDeviceGetAttribute(&h->c_sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->d_cbar == nullptr && (e = up(h, &h->d_cbar, std::vector<unsigned int>(2, 0u))) != cudaSuccess) return e;
  h->cs.bar = h->d_cbar;
  if ((e = build_sweeps(h, cf, h->cs, true, h->g_blocks, kSweepCoop, false)) != cudaSuccess) return e;
  h->c_nnz = h->cs.nnz;
  return cudaSuccess;
}

cudaError_t launch_coarse_solve(bddc_handle_s* h, const ApplyWork& W, const double* rc, double* uc, int nrhs,
                                cudaStream_t st, bool narrow) {
  if (h->n_c == 0) return cudaSuccess;
  cudaError_t e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  if (h->coarse_cg) {
    if (nrhs > kCgMaxRhs) return cudaErrorInvalidValue;
    CgArgs g{h->d_acp, h->d_acc, h->d_acv, rc, uc, W.cr, W.cy, W.cq, h->d_cgpart, h->d_cgiters,
             h->d_cbar, h->d_err, (int)h->n_c, nrhs, h->cg_maxit, h->cg_rtol, h->cbar_extra, h->cbar_cycles};
    if ((e = cudaMemsetAsync(h->d_cbar, 0, 2 * sizeof(unsigned int), st)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->c_sms);
    cfg.blockDim = dim3(narrow ? kCgThreadsNarrow : kCgThreadsWide);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_coarse_cg, g);
    h->launches++;
    return e;
  }
  return launch_sweeps(h, h->cs, rc, W.cr, W.cy, uc, nrhs, st, narrow, true);
}

cudaError_t launch_sweeps(bddc_handle_s* h, const SweepSet& S, const double* r, double* rp, double* y, double* u,
                          int nrhs, cudaStream_t st, bool narrow, bool inject) {
  if (S.n == 0) return cudaSuccess;
  if (nrhs > 1 && !S.multi) return cudaErrorInvalidValue;
  cudaError_t e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  const unsigned int extra = inject ? h->cbar_extra : 0u;
  const long long cycles = inject ? h->cbar_cycles : kBarrierWaitCycles;
  if (nrhs == 1 && S.block_form) {
    // heights below kmin: the per-level gather form (r' starts as a copy of
    // r, the backward sweeps read u by position); heights from kmin on: the
    // block form (fronts from r' and the block-form children)
    const int L = S.levels, kmin = std::max(0, std::min(S.block_min_height, L));
    auto level_phase = [&](int ph, bool fwd) {
      const SweepSet::LevelPhase& P = S.lv[ph];
      const int nblk = P.bb[kLevelClasses];
      if (nblk == 0) return;
      LevelArgs<double> la{S.seq + P.u0, S.gC, S.gI, fwd ? rp : y, fwd ? r : u, rp, y, u, (int)S.n, fwd ? 1 : 0,
                           {}, {}};
      std::memcpy(la.cb, P.cb, sizeof(la.cb));
      std::memcpy(la.bb, P.bb, sizeof(la.bb));
      k_level_sweep<double><<<nblk, kLevelThreads, 0, st>>>(la);
      h->launches++;
    };
    if (kmin > 0 &&
        (e = cudaMemcpyAsync(rp, r, sizeof(double) * S.n, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
    for (int ph = 0; ph < kmin; ++ph) level_phase(ph, true);
    for (int ph = kmin; ph < 2 * L - kmin; ++ph) {
      const int64_t k0 = S.bitem_off[ph], nblk = S.bitem_off[ph + 1] - k0;
      if (nblk == 0) continue;
      BlockArgs ba{S.bnodes, S.bkids, S.bcmap, S.bupd, S.bitems + k0, S.F, S.B, kmin > 0 ? rp : r, y, u, S.cbuf,
                   kmin};
      const int nbig = (int)S.bn_big[ph], nsmall = (int)nblk - nbig;
      const int grid = nbig + (nsmall + kBlockThreads / 32 - 1) / (kBlockThreads / 32);
      const size_t smem = (size_t)std::max(S.bphase_front[ph], nsmall > 0 ? (kBlockThreads / 32) * kSmallFront : 0) *
                          sizeof(double);
      if ((int)ph < S.levels)
        k_block_fwd<<<grid, kBlockThreads, smem, st>>>(ba, nbig, (int)nblk);
      else
        k_block_bwd<<<grid, kBlockThreads, smem, st>>>(ba, nbig, (int)nblk);
      h->launches++;
    }
    for (int ph = 2 * L - kmin; ph < 2 * L; ++ph) level_phase(ph, false);
    return cudaGetLastError();
  }
  if (nrhs == 1 && S.use_level && !S.lv.empty()) {
    // per-level form: one launch per phase, forward levels then backward
    // (the float32 form first rounds r into its copy: [r' | y | r] of x32)
    float* rp32 = S.gC32 ? S.x32 : nullptr;
    float* y32 = S.gC32 ? S.x32 + S.n : nullptr;
    float* r32 = S.gC32 ? S.x32 + 2 * S.n : nullptr;
    if (S.gC32 && S.n > 0) {
      const int grid = (int)std::min<int64_t>((S.n + 255) / 256, 4 * 1024);
      k_round_f32<<<grid, 256, 0, st>>>(r, r32, (int)S.n);
      h->launches++;
    }
    for (size_t ph = 0; ph < S.lv.size(); ++ph) {
      const SweepSet::LevelPhase& P = S.lv[ph];
      const int nblk = P.bb[kLevelClasses];
      if (nblk == 0) continue;
      const bool fwd = (int)ph < S.g_fwd;
      if (S.gC32) {
        LevelArgs<float> la{S.seq + P.u0, S.gC32, S.gI, fwd ? rp : y, fwd ? r : rp, rp, y, u, (int)S.n,
                            fwd ? 1 : 0, {}, {}};
        la.xa32 = fwd ? rp32 : y32;
        la.xb32 = fwd ? r32 : rp32;
        la.rp32 = rp32;
        la.y32 = y32;
        std::memcpy(la.cb, P.cb, sizeof(la.cb));
        std::memcpy(la.bb, P.bb, sizeof(la.bb));
        k_level_sweep<float><<<nblk, kLevelThreads, 0, st>>>(la);
      } else {
        LevelArgs<double> la{S.seq + P.u0, S.gC, S.gI, fwd ? rp : y, fwd ? r : rp, rp, y, u, (int)S.n,
                             fwd ? 1 : 0, {}, {}};
        std::memcpy(la.cb, P.cb, sizeof(la.cb));
        std::memcpy(la.bb, P.bb, sizeof(la.bb));
        k_level_sweep<double><<<nblk, kLevelThreads, 0, st>>>(la);
      }
      h->launches++;
    }
    return cudaGetLastError();
  }
  if ((e = cudaMemsetAsync(S.bar, 0, 2 * sizeof(unsigned int), st)) != cudaSuccess) return e;
  if (nrhs == 1 && S.gC) {
    const int sh = narrow ? 1 : 0;
    GatherArgs g{S.gU[sh], S.gwo[sh], S.gC, S.gI, r, rp, y, u, S.bar, h->d_err, S.g_fwd, (int)S.n, extra, cycles,
                 S.g_phases};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S.g_blocks);
    cfg.blockDim = dim3(narrow ? kGThreadsNarrow : kGThreadsWide);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = narrow ? cudaLaunchKernelEx(&cfg, k_coarse_sweeps<kGThreadsNarrow>, g)
               : cudaLaunchKernelEx(&cfg, k_coarse_sweeps<kGThreadsWide>, g);
    h->launches++;
    return e;
  }
  // row blocking pays from about 16 right-hand sides on (fewer, longer units
  // per level; measured on 10439 coarse dofs); the autotuner may move the
  // threshold
  const bool blocked = nrhs > 1 && nrhs >= h->tune_coarse_rb_min;
  CoarseArgs a{S.nodes, blocked ? S.units4 : S.units, S.list, S.upd, S.order, blocked ? S.lvl4 : S.lvl,
               S.F, S.B, r, rp, y, u, S.bar, h->d_err, S.levels, nrhs, extra, cycles};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(narrow ? h->c_sms : blocked ? S.grid4 : S.grid);
  cfg.blockDim = dim3((narrow || blocked) ? kThreads / 2 : kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = blocked ? cudaLaunchKernelEx(&cfg, k_coarse_solve<kRB>, a) : cudaLaunchKernelEx(&cfg, k_coarse_solve<1>, a);
  h->launches++;
  return e;
}

}  // namespace bddc
