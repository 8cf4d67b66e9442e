// Outer PCG kernels (sm_103a): the global SpMV with a precomputed Q1 stencil,
// the vector updates, and the dot products, each dot fused into the kernel
// that produces its operands. The per-column PCG scalars (alpha, beta, stop
// test) are updated by the last block of each reducing kernel, which sums the
// blocks' partial sums in a fixed order (deterministic, no float atomics).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace bddc {

namespace {

constexpr int kThreads = 256;

// Stencil offsets with a nonzero coupling, of which only the centre and the
// forward half are stored (A is symmetric: the coupling of node n to n - o is
// the forward coefficient of node n - o for offset o). 3D Q1: the centre, the
// 12 edge diagonals (two coordinates differ) and the 8 cube diagonals; the 6
// face neighbours couple with weight 0 for every sigma (the Q1 element
// matrix has a zero entry between nodes at Hamming distance 1). 2D: all 9
// points. Forward: a positive offset in node numbering (x fastest).
__constant__ int8_t c_fwd3[10][3] = {
    {-1, 1, 0}, {1, 1, 0}, {-1, 0, 1}, {1, 0, 1}, {0, -1, 1}, {0, 1, 1},
    {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}, {1, 1, 1}};
__constant__ int8_t c_fwd2[4][2] = {{1, 0}, {-1, 1}, {0, 1}, {1, 1}};

template <int DIM> struct Stencil;
template <> struct Stencil<3> { static constexpr int NH = 11; };   // centre + 10 forward offsets
template <> struct Stencil<2> { static constexpr int NH = 5; };

__device__ __forceinline__ bool on_boundary(int i, int ne) { return i == 0 || i == ne; }

template <int DIM>
__device__ __forceinline__ void fwd_offset(int s, int& dx, int& dy, int& dz) {
  dx = DIM == 3 ? c_fwd3[s][0] : c_fwd2[s][0];
  dy = DIM == 3 ? c_fwd3[s][1] : c_fwd2[s][1];
  dz = DIM == 3 ? c_fwd3[s][2] : 0;
}

// coef[s * ld + guard + n] = A[n, n + offset_s] for the centre (s = 0) and
// the forward offsets; zero on Dirichlet rows and for Dirichlet neighbours,
// and in the guard zones of `guard` entries before and after every array.
// A[n, m] = sum over the elements holding both nodes of sigma_e times the
// element-matrix entry for their Hamming distance.
template <int DIM>
__global__ void k_build_stencil(int ne, const double* __restrict__ sigma, double k0, double k1, double k2, double k3,
                                int64_t guard, double* __restrict__ coef) {
  constexpr int NH = Stencil<DIM>::NH;
  const int64_t n1 = ne + 1;
  const int64_t n_nodes = DIM == 2 ? n1 * n1 : n1 * n1 * n1;
  const int64_t ld = n_nodes + 2 * guard;
  const double kd[4] = {k0, k1, k2, k3};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NH * ld;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / ld);
    const int64_t nd = i - s * ld - guard;
    double c = 0.0;
    if (nd >= 0 && nd < n_nodes) {
      const int ix = (int)(nd % n1), iy = (int)((nd / n1) % n1), iz = DIM == 3 ? (int)(nd / (n1 * n1)) : 0;
      int dx = 0, dy = 0, dz = 0;
      if (s > 0) fwd_offset<DIM>(s - 1, dx, dy, dz);
      const int mx = ix + dx, my = iy + dy, mz = iz + dz;
      const bool dir = on_boundary(ix, ne) || on_boundary(iy, ne) || (DIM == 3 && on_boundary(iz, ne));
      const bool mdir = on_boundary(mx, ne) || on_boundary(my, ne) || (DIM == 3 && on_boundary(mz, ne));
      if (!dir && !mdir) {
        // elements with corner (ex, ey, ez) containing both nodes
        for (int ez = (DIM == 3 ? max(iz, mz) - 1 : 0); ez <= (DIM == 3 ? min(iz, mz) : 0); ++ez)
          for (int ey = max(iy, my) - 1; ey <= min(iy, my); ++ey)
            for (int ex = max(ix, mx) - 1; ex <= min(ix, mx); ++ex) {
              const int a = (ix - ex) | ((iy - ey) << 1) | (DIM == 3 ? (iz - ez) << 2 : 0);
              const int b = (mx - ex) | ((my - ey) << 1) | (DIM == 3 ? (mz - ez) << 2 : 0);
              const int64_t e = ex + (int64_t)ne * (ey + (int64_t)ne * ez);
              c += sigma[e] * kd[__popc(a ^ b)];
            }
      }
    }
    coef[i] = c;
  }
}

// Deterministic block reduction of up to three per-column sums. Thread t
// holds column k = t % nrhs; returns the block sums in red[slot][k]
// (valid for threads with t < nrhs after the call).
__device__ void block_reduce3(double s[3], int nrhs, double (*red)[kThreads]) {
  const int t = threadIdx.x;
  const int per = kThreads / nrhs;
  const int sub = t / nrhs, k = t - sub * nrhs;
  const bool live = t < per * nrhs;
  for (int q = 0; q < 3; ++q) red[q][t] = live ? s[q] : 0.0;
  __syncthreads();
  int P = 1;
  while (P * 2 <= per) P *= 2;
  if (live && sub >= P)
    for (int q = 0; q < 3; ++q) red[q][(sub - P) * nrhs + k] += red[q][t];
  __syncthreads();
  for (int st = P / 2; st > 0; st >>= 1) {
    if (live && sub < st)
      for (int q = 0; q < 3; ++q) red[q][t] += red[q][t + st * nrhs];
    __syncthreads();
  }
}

struct PcgState {
  double* scal;          // [S_COUNT][nrhs_max]
  int32_t* iscal;        // [I_COUNT][nrhs_max] + global flags
  double* partials;      // [blocks][3][nrhs]
  unsigned int* counter; // blocks done (reset by the last block)
  double* hist;          // [3][hist_cap + 1][nrhs_max]: ||r_k||, alpha_k, beta_k (null: not kept)
  int hist_cap;
  int nrhs_max;
  double rtol;
  int flexible;
};

// Iteration history: slot 0 = ||r_k|| (k = 0 .. iterations), 1 = alpha_k
// (k = 0 .. iterations - 1), 2 = beta_k, the beta computed after iteration
// k + 1 (k = 0 .. iterations - 2); entries beyond hist_cap are not kept.
__device__ __forceinline__ void hist_put(const PcgState& S, int slot, int it, int k, double v) {
  if (S.hist && it >= 0 && it <= S.hist_cap) S.hist[((int64_t)slot * (S.hist_cap + 1) + it) * S.nrhs_max + k] = v;
}

// Per-column PCG scalar update from the totals t[0..2] of column k.
__device__ void finalize_op(int op, int k, const double t[3], const PcgState& S, int* cnt, int* brk) {
  const int R = S.nrhs_max;
  double* rho = S.scal + S_RHO * R;
  double* alpha = S.scal + S_ALPHA * R;
  double* beta = S.scal + S_BETA * R;
  double* bb = S.scal + S_BB * R;
  double* rr = S.scal + S_RR * R;
  double* relres = S.scal + S_RELRES * R;
  int32_t* active = S.iscal + I_ACTIVE * R;
  int32_t* iters = S.iscal + I_ITERS * R;
  int32_t* status = S.iscal + I_STATUS * R;
  if (op == FIN_INIT) {            // t0 = b.b, t1 = r.r
    bb[k] = t[0]; rr[k] = t[1];
    const double bn = sqrt(t[0]), rn = sqrt(t[1]);
    relres[k] = bn > 0 ? rn / bn : 0.0;
    active[k] = (bn > 0 && !(rn <= S.rtol * bn)) ? 1 : 0;
    iters[k] = 0; status[k] = 0; alpha[k] = 0; beta[k] = 0;
    hist_put(S, 0, 0, k, rn);
    if (!isfinite(t[0]) || !isfinite(t[1])) {   // a non-finite right-hand side or start
      relres[k] = rn; active[k] = 0; status[k] = BDDC_ERR_BREAKDOWN; atomicAdd(brk, 1);
    }
  } else if (op == FIN_RHO) {      // t0 = r.z
    rho[k] = t[0];
  } else if (op == FIN_ALPHA) {    // t0 = p.q
    if (active[k]) {
      if (!(t[0] > 0.0) || !isfinite(t[0]) || !isfinite(rho[k])) {
        active[k] = 0; status[k] = BDDC_ERR_BREAKDOWN; alpha[k] = 0; atomicAdd(brk, 1);
      } else {
        alpha[k] = rho[k] / t[0];
        hist_put(S, 1, iters[k], k, alpha[k]);
      }
    } else {
      alpha[k] = 0;
    }
  } else if (op == FIN_CONV) {     // t0 = r.r
    if (active[k]) {
      iters[k] += 1;
      rr[k] = t[0];
      const double bn = sqrt(bb[k]), rn = sqrt(t[0]);
      relres[k] = rn / bn;
      hist_put(S, 0, iters[k], k, rn);
      if (rn <= S.rtol * bn) active[k] = 0;
      else if (!isfinite(rn)) { active[k] = 0; status[k] = BDDC_ERR_BREAKDOWN; atomicAdd(brk, 1); }
    }
  } else if (op == FIN_BETA) {     // t0 = r.z_new, t1 = r.z_old
    if (active[k]) {
      beta[k] = (S.flexible ? t[0] - t[1] : t[0]) / rho[k];
      rho[k] = t[0];
      hist_put(S, 2, iters[k] - 1, k, beta[k]);
    } else {
      beta[k] = 0;
    }
  }
  if (active[k]) atomicAdd(cnt, 1);
}

// Writes the block's partial sums; the last block to finish sums all
// partials in block order and applies finalize_op.
__device__ void reduce_and_finalize(double s[3], int nrhs, int op, const PcgState& S) {
  __shared__ double red[3][kThreads];
  __shared__ bool last;
  __shared__ int cnt, brk;
  block_reduce3(s, nrhs, red);
  const int t = threadIdx.x;
  if (t < nrhs)
    for (int q = 0; q < 3; ++q) S.partials[((int64_t)blockIdx.x * 3 + q) * nrhs + t] = red[q][t];
  __threadfence();
  __syncthreads();
  if (t == 0) last = atomicAdd(S.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // sum the partials of all blocks, fixed order
  const int per = kThreads / nrhs;
  const int sub = t / nrhs, k = t - sub * nrhs;
  double a[3] = {0, 0, 0};
  if (t < per * nrhs)
    for (int b = sub; b < (int)gridDim.x; b += per)
      for (int q = 0; q < 3; ++q) a[q] += __ldcg(&S.partials[((int64_t)b * 3 + q) * nrhs + k]);
  __syncthreads();
  block_reduce3(a, nrhs, red);
  if (t == 0) { cnt = 0; brk = 0; }
  __syncthreads();
  if (t < nrhs) {
    const double tot[3] = {red[0][t], red[1][t], red[2][t]};
    finalize_op(op, t, tot, S, &cnt, &brk);
  }
  __syncthreads();
  if (t == 0) {
    int32_t* flags = S.iscal + I_COUNT * S.nrhs_max;
    flags[0] = cnt;
    flags[1] = brk;
    *S.counter = 0;
  }
}

// y = A x with the precomputed half stencil; with op >= 0 also x.y per
// column and finalize_op(op). Thread t: column t % nrhs, nodes strided over
// the grid. Row n: the centre, A[n, n + o] = coef_o[n] and A[n, n - o] =
// coef_o[n - o] for every forward offset o; a neighbour index outside the
// vector is clamped into it and meets a zero coefficient (the guard zones,
// or the zero couplings of the boundary nodes there), so every row takes
// the same loads, none behind a branch.
template <int DIM>
__global__ void __launch_bounds__(kThreads, 4) k_spmv(int64_t n_nodes, int ne, int nrhs, int64_t guard,
                                                   const double* __restrict__ coef, const double* __restrict__ x,
                                                   double* __restrict__ y, int op, PcgState S) {
  constexpr int NH = Stencil<DIM>::NH;
  const int64_t n1 = ne + 1;
  const int64_t ld = n_nodes + 2 * guard;
  const double* c0 = coef + guard;
  const int per = kThreads / nrhs;
  const int sub = threadIdx.x / nrhs, k = threadIdx.x - sub * nrhs;
  double s[3] = {0, 0, 0};
  if (threadIdx.x < per * nrhs) {
    for (int64_t nd = blockIdx.x * (int64_t)per + sub; nd < n_nodes; nd += (int64_t)gridDim.x * per) {
      double part[4] = {__ldg(&c0[nd]) * __ldg(&x[nd * nrhs + k]), 0.0, 0.0, 0.0};
#pragma unroll
      for (int q = 1; q < NH; ++q) {
        int dx, dy, dz;
        fwd_offset<DIM>(q - 1, dx, dy, dz);
        const int64_t off = dx + n1 * (dy + n1 * dz);
        const int64_t up = min(nd + off, n_nodes - 1), dn = max(nd - off, (int64_t)0);
        const double* cq = c0 + (int64_t)q * ld;
        part[q & 3] = fma(__ldg(&cq[nd]), __ldg(&x[up * nrhs + k]), part[q & 3]);
        part[(q + 2) & 3] = fma(__ldg(&cq[nd - off]), __ldg(&x[dn * nrhs + k]), part[(q + 2) & 3]);
      }
      const double acc = (part[0] + part[1]) + (part[2] + part[3]);
      y[nd * nrhs + k] = acc;
      s[0] = fma(x[nd * nrhs + k], acc, s[0]);
    }
  }
  if (op >= 0) reduce_and_finalize(s, nrhs, op, S);
}

// x += alpha p; r -= alpha q; then r.r and the stop test (FIN_CONV)
__global__ void __launch_bounds__(kThreads) k_update_xr_conv(int64_t n_nodes, int nrhs, const double* __restrict__ p,
                                                             const double* __restrict__ q, double* __restrict__ x,
                                                             double* __restrict__ r, PcgState S) {
  const double* alpha = S.scal + S_ALPHA * S.nrhs_max;
  const int per = kThreads / nrhs;
  const int sub = threadIdx.x / nrhs, k = threadIdx.x - sub * nrhs;
  double s[3] = {0, 0, 0};
  if (threadIdx.x < per * nrhs) {
    const double a = alpha[k];
    for (int64_t nd = blockIdx.x * (int64_t)per + sub; nd < n_nodes; nd += (int64_t)gridDim.x * per) {
      const int64_t i = nd * nrhs + k;
      x[i] = fma(a, p[i], x[i]);
      const double ri = fma(-a, q[i], r[i]);
      r[i] = ri;
      s[0] = fma(ri, ri, s[0]);
    }
  }
  reduce_and_finalize(s, nrhs, FIN_CONV, S);
}

// Up to three dot products per column, then finalize_op(op).
__global__ void __launch_bounds__(kThreads) k_dots_fin(int64_t n_nodes, int nrhs, const double* __restrict__ a0,
                                                       const double* __restrict__ b0, const double* __restrict__ a1,
                                                       const double* __restrict__ b1, int op, PcgState S) {
  const int per = kThreads / nrhs;
  const int sub = threadIdx.x / nrhs, k = threadIdx.x - sub * nrhs;
  double s[3] = {0, 0, 0};
  if (threadIdx.x < per * nrhs) {
    for (int64_t nd = blockIdx.x * (int64_t)per + sub; nd < n_nodes; nd += (int64_t)gridDim.x * per) {
      const int64_t i = nd * nrhs + k;
      s[0] = fma(a0[i], b0[i], s[0]);
      if (a1) s[1] = fma(a1[i], b1[i], s[1]);
    }
  }
  reduce_and_finalize(s, nrhs, op, S);
}

PcgState state(bddc_handle_s* h, double rtol, int flexible) {
  return PcgState{h->d_scal, h->d_iscal, h->d_partials, h->d_counter, h->d_hist, h->hist_cap, h->nrhs_max, rtol,
                  flexible};
}

void stencil_coefs(int dim, double h, double c[4]) {
  if (dim == 2) { c[0] = 4.0 / 6; c[1] = -1.0 / 6; c[2] = -2.0 / 6; c[3] = 0; }
  else { c[0] = h / 3; c[1] = 0; c[2] = -h / 12; c[3] = -h / 12; }
}

}  // namespace

int stencil_points(int dim) { return dim == 3 ? Stencil<3>::NH : Stencil<2>::NH; }

int64_t stencil_guard(int dim, int ne) {
  const int64_t n1 = ne + 1;
  return dim == 3 ? n1 * n1 + n1 + 1 : n1 + 1;   // the largest forward offset
}

cudaError_t launch_build_stencil(bddc_handle_s* h, cudaStream_t st) {
  double c[4];
  stencil_coefs(h->dim, h->h, c);
  const int64_t guard = stencil_guard(h->dim, h->ne);
  const int64_t total = (int64_t)stencil_points(h->dim) * (h->n_nodes + 2 * guard);
  const int blocks = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, 1 << 20);
  if (h->dim == 3)
    k_build_stencil<3><<<blocks, kThreads, 0, st>>>(h->ne, h->d_sigma, c[0], c[1], c[2], c[3], guard, h->d_stencil);
  else
    k_build_stencil<2><<<blocks, kThreads, 0, st>>>(h->ne, h->d_sigma, c[0], c[1], c[2], c[3], guard, h->d_stencil);
  return cudaGetLastError();
}

cudaError_t launch_spmv(bddc_handle_s* h, const double* x, double* y, int nrhs, int op, double rtol, int flexible,
                        cudaStream_t st) {
  const PcgState S = state(h, rtol, flexible);
  const int64_t guard = stencil_guard(h->dim, h->ne);
  if (h->dim == 3)
    k_spmv<3><<<h->n_red_blocks, kThreads, 0, st>>>(h->n_nodes, h->ne, nrhs, guard, h->d_stencil, x, y, op, S);
  else
    k_spmv<2><<<h->n_red_blocks, kThreads, 0, st>>>(h->n_nodes, h->ne, nrhs, guard, h->d_stencil, x, y, op, S);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_update_xr_conv(bddc_handle_s* h, double* x, int nrhs, double rtol, int flexible,
                                  cudaStream_t st) {
  k_update_xr_conv<<<h->n_red_blocks, kThreads, 0, st>>>(h->n_nodes, nrhs, h->p_p, h->p_q, x, h->p_r,
                                                         state(h, rtol, flexible));
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_dots_fin(bddc_handle_s* h, int nrhs, const double* a0, const double* b0, const double* a1,
                            const double* b1, int op, double rtol, int flexible, cudaStream_t st) {
  k_dots_fin<<<h->n_red_blocks, kThreads, 0, st>>>(h->n_nodes, nrhs, a0, b0, a1, b1, op, state(h, rtol, flexible));
  h->launches++;
  return cudaGetLastError();
}

}  // namespace bddc
