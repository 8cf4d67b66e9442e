// Device kernels of the BDDC apply and of PCG (sm_103a).
//
// The apply computes M^-1 r = v1 + v2 + v3 (arXiv 2410.14786, Sec. 2) in the
// static-condensation form, which gives the same vector in exact arithmetic:
//   t_I   = A_II^-1 r_I                           (interior solves)
//   y'_G  = W r_G - A_GI t_I                       (condensed local right-hand side)
//   z_G   = K_GG y'_G,  g = Phi_G^T y'_G           (Eq. compzi on the interface; the
//                                                   coarse residual r_c = sum R_ci^T g)
//   u_c   = A_c^-1 r_c                             (Eq. coarsegrid)
//   v_G   = sum R^T W (z_G + Phi_G u_c)            (v1 + v2 on interface nodes)
//   z_I   = A_II^-1 (r_I - A_IG v_G)               (v1 + v2 + v3 on interior nodes:
//                                                   Eq. inner with r1 = r - A(v1+v2))
// The interior parts of z_i and of Phi_i R_ci u_c cancel in v1 + v2 + v3, so
// they are never formed. Dense operators are applied by one batched GEMV
// kernel; the rest are gathers over precomputed index maps (no atomics, so
// results are identical from run to run).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace bddc {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int threads = kThreads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 30));
}

// ---------------------------------------------------------------------------
// restriction: r_I (compact), W r_G (compact copies), zero Dirichlet outputs
// ---------------------------------------------------------------------------
__global__ void k_restrict(const double* __restrict__ r, int nrhs, const int32_t* __restrict__ inode,
                           int64_t nI, const int32_t* __restrict__ gnode, const double* __restrict__ gw,
                           int64_t nG, double* __restrict__ rI, double* __restrict__ yG,
                           const int32_t* __restrict__ dnode, int64_t nD, double* __restrict__ zout) {
  const int64_t total = (nI + nG + nD) * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = i / nrhs;
    int k = (int)(i - e * nrhs);
    if (e < nI) {
      rI[i] = r[(int64_t)inode[e] * nrhs + k];
    } else if (e < nI + nG) {
      int64_t q = e - nI;
      yG[q * nrhs + k] = gw[q] * r[(int64_t)gnode[q] * nrhs + k];
    } else if (zout) {
      zout[(int64_t)dnode[e - nI - nG] * nrhs + k] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// batched dense GEMV / skinny GEMM over row tiles of many operators
// ---------------------------------------------------------------------------
template <typename T> struct Elem;
template <> struct Elem<double> {
  static constexpr int V = 2;
  using Acc = double;
  __device__ static void load(const double* p, double out[2]) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    out[0] = v.x; out[1] = v.y;
  }
};
template <> struct Elem<float> {
  static constexpr int V = 4;
  using Acc = float;
  __device__ static void load(const float* p, float out[4]) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  }
};
template <> struct Elem<__nv_bfloat16> {
  static constexpr int V = 8;
  using Acc = float;
  __device__ static void load(const __nv_bfloat16* p, float out[8]) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      out[2 * i] = __uint_as_float(w[i] << 16);
      out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};

// Y[yoff + row, k] = sum_c Op[row, c] X[xoff + c, k] for the rows of one
// work item per block; columns k processed NRB at a time with the operand
// block staged in shared memory. With yscatter, row index j of Y becomes
// node yscatter[j] of a node-major vector.
template <typename T, int NRB>
__global__ void __launch_bounds__(kThreads) k_bgemv(const WorkItem* __restrict__ items,
                                                    const T* __restrict__ arena,
                                                    const double* __restrict__ X, double* __restrict__ Y,
                                                    const int32_t* __restrict__ yscatter, int nrhs) {
  using Acc = typename Elem<T>::Acc;
  constexpr int V = Elem<T>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* xs = reinterpret_cast<Acc*>(smem_raw);
  const WorkItem w = items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int rhs0 = 0; rhs0 < nrhs; rhs0 += NRB) {
    const int nr = min(NRB, nrhs - rhs0);
    if (rhs0) __syncthreads();
    for (int i = threadIdx.x; i < w.lda * NRB; i += blockDim.x) {
      const int c = i / NRB, k = i - c * NRB;
      double v = 0.0;
      if (c < w.ncols && k < nr) v = X[(int64_t)(w.xoff + c) * nrhs + rhs0 + k];
      xs[i] = (Acc)v;
    }
    __syncthreads();
    for (int rr = warp; rr < w.nrows; rr += nw) {
      const int row = w.row0 + rr;
      const T* a = arena + w.moff + (int64_t)row * w.lda;
      Acc acc[NRB];
#pragma unroll
      for (int k = 0; k < NRB; ++k) acc[k] = Acc(0);
#pragma unroll 4
      for (int c0 = lane * V; c0 < w.lda; c0 += 32 * V) {
        Acc av[V];
        Elem<T>::load(a + c0, av);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int k = 0; k < NRB; ++k) acc[k] = fma(av[v], xs[(c0 + v) * NRB + k], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < NRB; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
      double out = 0.0;
#pragma unroll
      for (int k = 0; k < NRB; ++k)
        if (lane == k) out = (double)acc[k];
      if (lane < nr) {
        const int64_t j = (int64_t)w.yoff + row;
        const int64_t dst = yscatter ? (int64_t)yscatter[j] : j;
        Y[dst * nrhs + rhs0 + lane] = out;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// y'_G = W r_G - A_GI t_I   (rows: interface copies; cols: compact interior)
// ---------------------------------------------------------------------------
__global__ void k_iface_rhs(int64_t nG, int nrhs, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ val,
                            const double* __restrict__ tI, double* __restrict__ yG) {
  const int64_t total = nG * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = i / nrhs;
    const int k = (int)(i - q * nrhs);
    double s = 0.0;
    for (int j = ptr[q]; j < ptr[q + 1]; ++j) s = fma(val[j], tI[(int64_t)col[j] * nrhs + k], s);
    yG[i] -= s;
  }
}

// g[pos, k] = sum_l Phi_G^T[c, l] y'_G[l, k] (one warp per local constraint)
__global__ void k_coarse_local(int64_t nC, int nrhs, const int32_t* __restrict__ csub,
                               const int32_t* __restrict__ coff, const int32_t* __restrict__ goff,
                               const int64_t* __restrict__ phit_off, const double* __restrict__ phit,
                               const double* __restrict__ yG, double* __restrict__ g) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nC) return;
  const int s = csub[wid];
  const int c = (int)(wid - coff[s]);
  const int g0 = goff[s], nG = goff[s + 1] - g0;
  const double* row = phit + phit_off[s] + (int64_t)c * nG;
  for (int k = 0; k < nrhs; ++k) {
    double acc = 0.0;
    for (int l = lane; l < nG; l += 32) acc = fma(row[l], yG[(int64_t)(g0 + l) * nrhs + k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) g[wid * nrhs + k] = acc;
  }
}

// r_c[c, k] = sum over the local constraints that map to coarse dof c
__global__ void k_coarse_gather(int64_t n_c, int nrhs, const int32_t* __restrict__ ptr,
                                const int32_t* __restrict__ idx, const double* __restrict__ g,
                                double* __restrict__ rc) {
  const int64_t total = n_c * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / nrhs;
    const int k = (int)(i - c * nrhs);
    double s = 0.0;
    for (int j = ptr[c]; j < ptr[c + 1]; ++j) s += g[(int64_t)idx[j] * nrhs + k];
    rc[i] = s;
  }
}

// z[node] = sum over the copies q of the node: W_q (z_G[q] + Phi_G[q, :] u_c[R_c])
__global__ void k_prolong(int64_t n_gu, int nrhs, const int32_t* __restrict__ gu_node,
                          const int32_t* __restrict__ gu_ptr, const int32_t* __restrict__ gu_copy,
                          const double* __restrict__ gw, const double* __restrict__ zG,
                          const int64_t* __restrict__ phirow, const int32_t* __restrict__ gsub,
                          const int32_t* __restrict__ coff, const int32_t* __restrict__ ccdof,
                          const double* __restrict__ phi, const double* __restrict__ uc,
                          double* __restrict__ z) {
  const int64_t total = n_gu * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = i / nrhs;
    const int k = (int)(i - u * nrhs);
    double v = 0.0;
    for (int j = gu_ptr[u]; j < gu_ptr[u + 1]; ++j) {
      const int q = gu_copy[j];
      const int s = gsub[q];
      const int c0 = coff[s], nc = coff[s + 1] - c0;
      const double* prow = phi + phirow[q];
      double e = zG[(int64_t)q * nrhs + k];
      for (int c = 0; c < nc; ++c) e = fma(prow[c], uc[(int64_t)ccdof[c0 + c] * nrhs + k], e);
      v = fma(gw[q], e, v);
    }
    z[(int64_t)gu_node[u] * nrhs + k] = v;
  }
}

// b_I = r_I - A_IG v_G   (rows: compact interior; cols: node ids)
__global__ void k_interior_rhs(int64_t nI, int nrhs, const int32_t* __restrict__ ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val,
                               const double* __restrict__ rI, const double* __restrict__ z,
                               double* __restrict__ bI) {
  const int64_t total = nI * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / nrhs;
    const int k = (int)(i - p * nrhs);
    double s = rI[i];
    for (int j = ptr[p]; j < ptr[p + 1]; ++j) s = fma(-val[j], z[(int64_t)col[j] * nrhs + k], s);
    bI[i] = s;
  }
}

// zero the interface and Dirichlet entries of a vector
__global__ void k_zero_nodes(int64_t n, int nrhs, const int32_t* __restrict__ nodes, double* __restrict__ x) {
  const int64_t total = n * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / nrhs;
    x[(int64_t)nodes[e] * nrhs + (i - e * nrhs)] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// matrix-free Q1 operators on the structured grid
// ---------------------------------------------------------------------------
// coef[d] = entry of the element matrix between local nodes at Hamming distance d
template <int DIM>
__global__ void k_q1_apply(int ne, int nrhs, const double* __restrict__ sigma, double c0, double c1,
                           double c2, double c3, int use_sigma, int skip_dirichlet_cols,
                           const double* __restrict__ x, double* __restrict__ y) {
  const int64_t n1 = ne + 1;
  const int64_t n_nodes = DIM == 2 ? n1 * n1 : n1 * n1 * n1;
  const double coef[4] = {c0, c1, c2, c3};
  for (int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; nd < n_nodes;
       nd += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(nd % n1), iy = (int)((nd / n1) % n1), iz = DIM == 3 ? (int)(nd / (n1 * n1)) : 0;
    const bool dir = ix == 0 || ix == ne || iy == 0 || iy == ne || (DIM == 3 && (iz == 0 || iz == ne));
    for (int k = 0; k < nrhs; ++k) {
      double acc = 0.0;
      if (!dir) {
#pragma unroll
        for (int ez_ = 0; ez_ < (DIM == 3 ? 2 : 1); ++ez_) {
#pragma unroll
          for (int ey_ = 0; ey_ < 2; ++ey_) {
#pragma unroll
            for (int ex_ = 0; ex_ < 2; ++ex_) {
              const int ex = ix - 1 + ex_, ey = iy - 1 + ey_, ez = DIM == 3 ? iz - 1 + ez_ : 0;
              if (ex < 0 || ex >= ne || ey < 0 || ey >= ne || ez < 0 || (DIM == 3 && ez >= ne)) continue;
              const int a = (1 - ex_) | ((1 - ey_) << 1) | (DIM == 3 ? (1 - ez_) << 2 : 0);
              const int64_t e = ex + (int64_t)ne * (ey + (int64_t)ne * ez);
              double s = 0.0;
#pragma unroll
              for (int b = 0; b < (1 << DIM); ++b) {
                const int bx = ex + (b & 1), by = ey + ((b >> 1) & 1), bz = DIM == 3 ? ez + ((b >> 2) & 1) : 0;
                if (skip_dirichlet_cols &&
                    (bx == 0 || bx == ne || by == 0 || by == ne || (DIM == 3 && (bz == 0 || bz == ne))))
                  continue;
                const double cf = coef[__popc(a ^ b)];
                if (cf == 0.0) continue;
                s = fma(cf, x[(bx + n1 * (by + n1 * (int64_t)bz)) * nrhs + k], s);
              }
              acc = use_sigma ? fma(sigma[e], s, acc) : acc + s;
            }
          }
        }
      }
      y[nd * nrhs + k] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// PCG vector kernels
// ---------------------------------------------------------------------------
// per-column partial sums; block b writes partials[(b * 3 + slot) * nrhs + k]
__global__ void k_dots(int64_t n_nodes, int nrhs, const double* __restrict__ a0, const double* __restrict__ b0,
                       const double* __restrict__ a1, const double* __restrict__ b1,
                       const double* __restrict__ a2, const double* __restrict__ b2,
                       double* __restrict__ partials) {
  __shared__ double red[3][kThreads];
  const int per = kThreads / nrhs;         // nodes per block step
  const int tid = threadIdx.x;
  const bool live = tid < per * nrhs;
  const int k = tid % nrhs, sub = tid / nrhs;
  double s0 = 0, s1 = 0, s2 = 0;
  if (live) {
    for (int64_t nd = blockIdx.x * (int64_t)per + sub; nd < n_nodes; nd += (int64_t)gridDim.x * per) {
      const int64_t i = nd * nrhs + k;
      s0 = fma(a0[i], b0[i], s0);
      if (a1) s1 = fma(a1[i], b1[i], s1);
      if (a2) s2 = fma(a2[i], b2[i], s2);
    }
  }
  red[0][tid] = s0; red[1][tid] = s1; red[2][tid] = s2;
  __syncthreads();
  if (tid < nrhs) {
    double t0 = 0, t1 = 0, t2 = 0;
    for (int j = 0; j < per; ++j) {
      t0 += red[0][j * nrhs + tid];
      t1 += red[1][j * nrhs + tid];
      t2 += red[2][j * nrhs + tid];
    }
    partials[(blockIdx.x * 3 + 0) * nrhs + tid] = t0;
    partials[(blockIdx.x * 3 + 1) * nrhs + tid] = t1;
    partials[(blockIdx.x * 3 + 2) * nrhs + tid] = t2;
  }
}

__global__ void k_finalize(int op, int nrhs, int nblocks, const double* __restrict__ partials,
                           double* __restrict__ scal, int32_t* __restrict__ iscal, int nrhs_max,
                           double rtol, int flexible) {
  const int k = threadIdx.x;
  double t[3] = {0, 0, 0};
  if (k < nrhs)
    for (int b = 0; b < nblocks; ++b)
      for (int s = 0; s < 3; ++s) t[s] += partials[(b * 3 + s) * nrhs + k];
  double* rho = scal + S_RHO * nrhs_max;
  double* alpha = scal + S_ALPHA * nrhs_max;
  double* beta = scal + S_BETA * nrhs_max;
  double* bb = scal + S_BB * nrhs_max;
  double* rr = scal + S_RR * nrhs_max;
  double* relres = scal + S_RELRES * nrhs_max;
  int32_t* active = iscal + I_ACTIVE * nrhs_max;
  int32_t* iters = iscal + I_ITERS * nrhs_max;
  int32_t* status = iscal + I_STATUS * nrhs_max;
  int32_t* flags = iscal + I_COUNT * nrhs_max;      // [0] active count, [1] breakdown
  __shared__ int cnt, brk;
  if (k == 0) { cnt = 0; brk = 0; }
  __syncthreads();
  if (k < nrhs) {
    if (op == FIN_INIT) {            // t0 = b.b, t1 = r.r
      bb[k] = t[0]; rr[k] = t[1];
      const double bn = sqrt(t[0]), rn = sqrt(t[1]);
      relres[k] = bn > 0 ? rn / bn : 0.0;
      active[k] = (bn > 0 && !(rn <= rtol * bn)) ? 1 : 0;
      iters[k] = 0; status[k] = 0;
      alpha[k] = 0; beta[k] = 0;
    } else if (op == FIN_RHO) {      // t0 = r.z
      rho[k] = t[0];
    } else if (op == FIN_ALPHA) {    // t0 = p.q
      if (active[k]) {
        if (!(t[0] > 0.0) || !isfinite(t[0]) || !isfinite(rho[k])) {
          active[k] = 0; status[k] = BDDC_ERR_BREAKDOWN; alpha[k] = 0; atomicAdd(&brk, 1);
        } else {
          alpha[k] = rho[k] / t[0];
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
        if (rn <= rtol * bn) active[k] = 0;
        else if (!isfinite(rn)) { active[k] = 0; status[k] = BDDC_ERR_BREAKDOWN; atomicAdd(&brk, 1); }
      }
    } else if (op == FIN_BETA) {     // t0 = r.z_new, t1 = r.z_old
      if (active[k]) {
        const double num = flexible ? t[0] - t[1] : t[0];
        beta[k] = num / rho[k];
        rho[k] = t[0];
      } else {
        beta[k] = 0;
      }
    }
    if (active[k]) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (k == 0) { flags[0] = cnt; flags[1] = brk; }
}

__global__ void k_update_xr(int64_t n, int nrhs, const double* __restrict__ alpha, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const int64_t total = n * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = alpha[i % nrhs];
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}

__global__ void k_update_p(int64_t n, int nrhs, const double* __restrict__ beta, const double* __restrict__ z,
                           double* __restrict__ p, double* __restrict__ zold) {
  const int64_t total = n * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = z[i];
    p[i] = fma(beta[i % nrhs], p[i], zi);
    zold[i] = zi;
  }
}

__global__ void k_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                           double* __restrict__ r, double* __restrict__ zero_a, double* __restrict__ zero_b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = b[i] - q[i];
    zero_a[i] = 0.0;
    zero_b[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t bgemv_t(const WorkItem* items, int n_items, int max_lda, const void* arena, const double* X,
                    double* Y, const int32_t* yscatter, int nrhs, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  using Acc = typename Elem<T>::Acc;
  const T* A = static_cast<const T*>(arena);
  auto run = [&](auto kern, int nrb) -> cudaError_t {
    size_t sm = (size_t)max_lda * nrb * sizeof(Acc);
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    kern<<<n_items, kThreads, sm, st>>>(items, A, X, Y, yscatter, nrhs);
    return cudaGetLastError();
  };
  const size_t limit = 200 * 1024;
  if (nrhs >= 8 && (size_t)max_lda * 8 * sizeof(Acc) <= limit) return run(k_bgemv<T, 8>, 8);
  if (nrhs >= 4 && (size_t)max_lda * 4 * sizeof(Acc) <= limit) return run(k_bgemv<T, 4>, 4);
  if (nrhs >= 2 && (size_t)max_lda * 2 * sizeof(Acc) <= limit) return run(k_bgemv<T, 2>, 2);
  return run(k_bgemv<T, 1>, 1);
}

cudaError_t bgemv(int precision, const WorkItem* items, int n_items, int max_lda, const void* arena,
                  const double* X, double* Y, const int32_t* yscatter, int nrhs, cudaStream_t st) {
  switch (precision) {
    case BDDC_PREC_FP64: return bgemv_t<double>(items, n_items, max_lda, arena, X, Y, yscatter, nrhs, st);
    case BDDC_PREC_FP32: return bgemv_t<float>(items, n_items, max_lda, arena, X, Y, yscatter, nrhs, st);
    default: return bgemv_t<__nv_bfloat16>(items, n_items, max_lda, arena, X, Y, yscatter, nrhs, st);
  }
}

}  // namespace

cudaError_t launch_interior_correction(bddc_handle_s* h, const double* b, double* x, int nrhs,
                                       cudaStream_t st) {
  // x = 0 on interface and Dirichlet nodes, A_II^-1 b_I on interior nodes
  k_restrict<<<blocks_for(h->nI_tot * nrhs), kThreads, 0, st>>>(b, nrhs, h->d_inode, h->nI_tot, nullptr,
                                                                nullptr, 0, h->w_rI, nullptr, h->d_dnode,
                                                                h->n_dir, x);
  if (h->n_gu)
    k_zero_nodes<<<blocks_for(h->n_gu * nrhs), kThreads, 0, st>>>(h->n_gu, nrhs, h->d_gu_node, x);
  cudaError_t e = bgemv(h->precision, h->d_wi_I, h->n_wi_I, h->max_cols_I, h->d_aii, h->w_rI, x,
                        h->d_inode, nrhs, st);
  h->launches += 1 + (h->n_gu > 0) + (h->n_wi_I > 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_apply(bddc_handle_s* h, const double* r, double* z, int nrhs, cudaStream_t st,
                         cudaEvent_t* ev) {
  cudaError_t e;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], st);
  };
  mark(0);
  // restriction + zero Dirichlet entries of z
  const int64_t tot = (h->nI_tot + h->nG_tot + h->n_dir) * nrhs;
  k_restrict<<<blocks_for(tot), kThreads, 0, st>>>(r, nrhs, h->d_inode, h->nI_tot, h->d_gnode, h->d_gw,
                                                   h->nG_tot, h->w_rI, h->w_yG, h->d_dnode, h->n_dir, z);
  h->launches++;
  mark(1);
  // t_I = A_II^-1 r_I
  if ((e = bgemv(h->precision, h->d_wi_I, h->n_wi_I, h->max_cols_I, h->d_aii, h->w_rI, h->w_tI, nullptr,
                 nrhs, st)) != cudaSuccess)
    return e;
  h->launches += h->n_wi_I > 0;
  mark(2);
  if (h->nG_tot) {
    // y'_G = W r_G - A_GI t_I; z_G = K_GG y'_G
    k_iface_rhs<<<blocks_for(h->nG_tot * nrhs), kThreads, 0, st>>>(h->nG_tot, nrhs, h->d_agi_ptr,
                                                                   h->d_agi_col, h->d_agi_val, h->w_tI,
                                                                   h->w_yG);
    h->launches++;
  }
  mark(3);
  if (h->nG_tot) {
    if ((e = bgemv(h->precision, h->d_wi_G, h->n_wi_G, h->max_cols_G, h->d_kgg, h->w_yG, h->w_zG, nullptr,
                   nrhs, st)) != cudaSuccess)
      return e;
    h->launches++;
  }
  mark(4);
  if (h->n_c) {
    // coarse residual r_c = sum R_ci^T Phi_G^T y'_G
    k_coarse_local<<<blocks_for(h->nC_tot * 32), kThreads, 0, st>>>(h->nC_tot, nrhs, h->d_csub, h->d_sub_coff,
                                                                    h->d_sub_goff, h->d_sub_phit_off, h->d_phit,
                                                                    h->w_yG, h->w_g);
    k_coarse_gather<<<blocks_for(h->n_c * nrhs), kThreads, 0, st>>>(h->n_c, nrhs, h->d_cg_ptr, h->d_cg_idx,
                                                                    h->w_g, h->w_rc);
    h->launches += 2;
  }
  mark(5);
  if (h->n_c) {
    // u_c = A_c^-1 r_c
    if ((e = bgemv(BDDC_PREC_FP64, h->d_wi_C, h->n_wi_C, h->ldc, h->d_acinv, h->w_rc, h->w_uc, nullptr, nrhs,
                   st)) != cudaSuccess)
      return e;
    h->launches++;
  }
  mark(6);
  if (h->n_gu) {
    k_prolong<<<blocks_for(h->n_gu * nrhs), kThreads, 0, st>>>(h->n_gu, nrhs, h->d_gu_node, h->d_gu_ptr,
                                                               h->d_gu_copy, h->d_gw, h->w_zG, h->d_gcopy_phirow,
                                                               h->d_gcopy_sub, h->d_sub_coff, h->d_ccdof,
                                                               h->d_phi, h->w_uc, z);
    h->launches++;
  }
  mark(7);
  // z_I = A_II^-1 (r_I - A_IG v_G)
  k_interior_rhs<<<blocks_for(h->nI_tot * nrhs), kThreads, 0, st>>>(h->nI_tot, nrhs, h->d_aig_ptr,
                                                                    h->d_aig_col, h->d_aig_val, h->w_rI, z,
                                                                    h->w_bI);
  h->launches++;
  mark(8);
  if ((e = bgemv(h->precision, h->d_wi_I, h->n_wi_I, h->max_cols_I, h->d_aii, h->w_bI, z, h->d_inode, nrhs,
                 st)) != cudaSuccess)
    return e;
  h->launches += h->n_wi_I > 0;
  mark(9);
  return cudaGetLastError();
}

static void q1_coefs(int dim, double h, bool mass, double c[4]) {
  if (!mass) {
    if (dim == 2) { c[0] = 4.0 / 6; c[1] = -1.0 / 6; c[2] = -2.0 / 6; c[3] = 0; }
    else { c[0] = h / 3; c[1] = 0; c[2] = -h / 12; c[3] = -h / 12; }
  } else {
    if (dim == 2) { const double s = h * h / 36; c[0] = 4 * s; c[1] = 2 * s; c[2] = s; c[3] = 0; }
    else { const double s = h * h * h / 216; c[0] = 8 * s; c[1] = 4 * s; c[2] = 2 * s; c[3] = s; }
  }
}

cudaError_t launch_matvec(bddc_handle_s* h, const double* x, double* y, int nrhs, cudaStream_t st) {
  double c[4];
  q1_coefs(h->dim, h->h, false, c);
  if (h->dim == 2)
    k_q1_apply<2><<<blocks_for(h->n_nodes), kThreads, 0, st>>>(h->ne, nrhs, h->d_sigma, c[0], c[1], c[2], c[3],
                                                               1, 1, x, y);
  else
    k_q1_apply<3><<<blocks_for(h->n_nodes), kThreads, 0, st>>>(h->ne, nrhs, h->d_sigma, c[0], c[1], c[2], c[3],
                                                               1, 1, x, y);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_rhs(bddc_handle_s* h, const double* f, double* b, int nrhs, cudaStream_t st) {
  double c[4];
  q1_coefs(h->dim, h->h, true, c);
  if (h->dim == 2)
    k_q1_apply<2><<<blocks_for(h->n_nodes), kThreads, 0, st>>>(h->ne, nrhs, nullptr, c[0], c[1], c[2], c[3], 0,
                                                               0, f, b);
  else
    k_q1_apply<3><<<blocks_for(h->n_nodes), kThreads, 0, st>>>(h->ne, nrhs, nullptr, c[0], c[1], c[2], c[3], 0,
                                                               0, f, b);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_dots(bddc_handle_s* h, int nrhs, const double* a0, const double* b0, const double* a1,
                        const double* b1, const double* a2, const double* b2, cudaStream_t st) {
  k_dots<<<h->n_red_blocks, kThreads, 0, st>>>(h->n_nodes, nrhs, a0, b0, a1, b1, a2, b2, h->d_partials);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_finalize(bddc_handle_s* h, int op, int nrhs, double rtol, int flexible, cudaStream_t st) {
  k_finalize<<<1, 64, 0, st>>>(op, nrhs, h->n_red_blocks, h->d_partials, h->d_scal, h->d_iscal, h->nrhs_max,
                               rtol, flexible);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_update_xr(bddc_handle_s* h, double* x, int nrhs, cudaStream_t st) {
  k_update_xr<<<blocks_for(h->n_nodes * nrhs), kThreads, 0, st>>>(h->n_nodes, nrhs, h->d_scal + S_ALPHA * h->nrhs_max,
                                                                  h->p_p, h->p_q, x, h->p_r);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_update_p(bddc_handle_s* h, int nrhs, cudaStream_t st) {
  k_update_p<<<blocks_for(h->n_nodes * nrhs), kThreads, 0, st>>>(h->n_nodes, nrhs, h->d_scal + S_BETA * h->nrhs_max,
                                                                 h->p_z, h->p_p, h->p_zold);
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_residual(bddc_handle_s* h, const double* b, int nrhs, cudaStream_t st) {
  const int64_t n = h->n_nodes * nrhs;
  k_residual<<<blocks_for(n), kThreads, 0, st>>>(n, b, h->p_q, h->p_r, h->p_p, h->p_zold);
  h->launches++;
  return cudaGetLastError();
}

}  // namespace bddc
