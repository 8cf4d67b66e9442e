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
// ONE: a single right-hand side (nrhs = 1 at compile time: no index division).
template <bool ONE>
__global__ void k_restrict(const double* __restrict__ r, int nrhs_, const int32_t* __restrict__ inode,
                           int64_t nI, const int32_t* __restrict__ gnode, const double* __restrict__ gw,
                           int64_t nG, double* __restrict__ rI, double* __restrict__ yG,
                           const int32_t* __restrict__ dnode, int64_t nD, double* __restrict__ zout) {
  const int nrhs = ONE ? 1 : nrhs_;
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
// One thread per (row, block of CB columns; CB = 1 measured fastest for 1 to
// 64 columns: more threads hide more latency), the CSR loop unrolled so that
// the loads of several nonzeros are in flight together.
// y'_G = W r_G - A_GI t_I (rows: interface copies; cols: compact interior).
template <int CB, bool ONE>
__global__ void k_iface_rhs(int64_t nG, int nrhs_, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ col, const double* __restrict__ val,
                            const double* __restrict__ tI, const int32_t* __restrict__ gnode,
                            const double* __restrict__ gw, const double* __restrict__ r, double* __restrict__ yG) {
  const int nrhs = ONE ? 1 : nrhs_;
  const int ncb = (nrhs + CB - 1) / CB;
  const int64_t total = nG * ncb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / ncb;
    const int kb = (int)(t - q * ncb) * CB;
    double s[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) s[c] = 0.0;
    const int j1 = ptr[q + 1];
#pragma unroll 4
    for (int j = ptr[q]; j < j1; ++j) {
      const double v = val[j];
      const double* tp = tI + (int64_t)col[j] * nrhs + kb;
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (kb + c < nrhs) s[c] = fma(v, tp[c], s[c]);
    }
    double* yp = yG + q * nrhs + kb;
    const double* rp = r + (int64_t)gnode[q] * nrhs + kb;
    const double w = gw[q];
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (kb + c < nrhs) yp[c] = w * rp[c] - s[c];
  }
}

// r_c[c, k] = sum over the local constraints that map to coarse dof c
template <bool ONE>
__global__ void k_coarse_gather(int64_t n_c, int nrhs_, const int32_t* __restrict__ ptr,
                                const int32_t* __restrict__ idx, const double* __restrict__ g,
                                double* __restrict__ rc) {
  const int nrhs = ONE ? 1 : nrhs_;
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

// u_c per local constraint (the values Phi_G multiplies in the prolongation)
__global__ void k_gather_rows(int64_t n, int nrhs, const int32_t* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * nrhs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nrhs;
    dst[i] = src[(int64_t)perm[r] * nrhs + (i - r * nrhs)];
  }
}

// z rows of the compact interior result: dst[perm[i]] = src[i]
template <bool ONE>
__global__ void k_scatter_rows(int64_t n, int nrhs_, const int32_t* __restrict__ perm, const double* __restrict__ src,
                               double* __restrict__ dst) {
  const int nrhs = ONE ? 1 : nrhs_;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * nrhs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nrhs;
    dst[(int64_t)perm[r] * nrhs + (i - r * nrhs)] = src[i];
  }
}

// e_G = Phi_G u_c per interface copy, read from the Phi_G^T array of the
// coarse residual (n_ci rows of n_Gi entries per subdomain): one block per
// subdomain stages the subdomain's coarse values u_c[R_ci] in shared memory,
// thread `col` owns interface copy col and sums over the n_ci rows (loads
// coalesced across the threads). Columns of u_c in chunks of NB.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) k_phi_prolong(int n_sub, int nrhs, const T* __restrict__ pt,
                                                         const int64_t* __restrict__ pt_off,
                                                         const int32_t* __restrict__ pt_ld,
                                                         const int32_t* __restrict__ goff,
                                                         const int32_t* __restrict__ coff,
                                                         const int32_t* __restrict__ ccdof,
                                                         const double* __restrict__ uc, double* __restrict__ eG) {
  using Acc = typename Elem<T>::Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* us = reinterpret_cast<Acc*>(smem_raw);     // [n_ci][nrhs]
  for (int s = blockIdx.x; s < n_sub; s += gridDim.x) {
    const int g0 = goff[s], nG = goff[s + 1] - g0, c0 = coff[s], nc = coff[s + 1] - c0;
    __syncthreads();
    for (int i = threadIdx.x; i < nc * nrhs; i += blockDim.x) {
      const int j = i / nrhs, k = i - j * nrhs;
      us[i] = (Acc)uc[(int64_t)ccdof[c0 + j] * nrhs + k];
    }
    __syncthreads();
    const T* a = pt + pt_off[s];
    const int64_t ld = pt_ld[s];
    for (int col = threadIdx.x; col < nG; col += blockDim.x)
      for (int kb = 0; kb < nrhs; kb += NB) {
        Acc acc[NB];
#pragma unroll
        for (int kk = 0; kk < NB; ++kk) acc[kk] = Acc(0);
        for (int j = 0; j < nc; ++j) {
          const Acc v = (Acc)__ldg(a + j * ld + col);
#pragma unroll
          for (int kk = 0; kk < NB; ++kk)
            if (NB == 1 || kb + kk < nrhs) acc[kk] = fma(v, us[j * nrhs + kb + kk], acc[kk]);
        }
        double* out = eG + (int64_t)(g0 + col) * nrhs + kb;
#pragma unroll
        for (int kk = 0; kk < NB; ++kk)
          if (NB == 1 || kb + kk < nrhs) out[kk] = (double)acc[kk];
      }
  }
}

// z[node] = sum over the copies q of the node of W_q (z_G[q] + (Phi_G u_c)[q])
// (and z = 0 at the Dirichlet nodes dnode[0 .. nD))
template <int CB, bool ONE>
__global__ void k_prolong_gather(int64_t n_gu, int nrhs_, const int32_t* __restrict__ gu_node,
                                 const int32_t* __restrict__ gu_ptr, const int32_t* __restrict__ gu_copy,
                                 const double* __restrict__ gw, const double* __restrict__ zG,
                                 const double* __restrict__ eG, double* __restrict__ z,
                                 const int32_t* __restrict__ dnode, int64_t nD) {
  const int nrhs = ONE ? 1 : nrhs_;
  const int ncb = (nrhs + CB - 1) / CB;
  const int64_t total = n_gu * ncb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nD * nrhs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / nrhs;
    z[(int64_t)dnode[e] * nrhs + (i - e * nrhs)] = 0.0;
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = t / ncb;
    const int kb = (int)(t - u * ncb) * CB;
    double v[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) v[c] = 0.0;
    const int j1 = gu_ptr[u + 1];
#pragma unroll 4
    for (int j = gu_ptr[u]; j < j1; ++j) {
      const int32_t cq = gu_copy[j];
      const double w = gw[cq];
      const int64_t q = (int64_t)cq * nrhs + kb;
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (kb + c < nrhs) v[c] = fma(w, zG[q + c] + eG[q + c], v[c]);
    }
    double* zp = z + (int64_t)gu_node[u] * nrhs + kb;
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (kb + c < nrhs) zp[c] = v[c];
  }
}

// b_I = r_I - A_IG v_G   (rows: compact interior; cols: node ids)
template <int CB, bool ONE>
__global__ void k_interior_rhs(int64_t nI, int nrhs_, const int32_t* __restrict__ ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val,
                               const int32_t* __restrict__ inode, const double* __restrict__ r,
                               const double* __restrict__ z, double* __restrict__ bI) {
  const int nrhs = ONE ? 1 : nrhs_;
  const int ncb = (nrhs + CB - 1) / CB;
  const int64_t total = nI * ncb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / ncb;
    const int kb = (int)(t - p * ncb) * CB;
    const double* rp = r + (int64_t)inode[p] * nrhs + kb;
    double s[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) s[c] = kb + c < nrhs ? rp[c] : 0.0;
    const int j1 = ptr[p + 1];
#pragma unroll 4
    for (int j = ptr[p]; j < j1; ++j) {
      const double v = val[j];
      const double* zp = z + (int64_t)col[j] * nrhs + kb;
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (kb + c < nrhs) s[c] = fma(-v, zp[c], s[c]);
    }
    double* bp = bI + p * nrhs + kb;
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (kb + c < nrhs) bp[c] = s[c];
  }
}

// u_c = sum of the per-panel partial products of A_c^-1 r_c
__global__ void k_panel_sum(int64_t n, int npanels, const double* __restrict__ part, double* __restrict__ uc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < npanels; ++p) s += part[(int64_t)p * n + i];
    uc[i] = s;
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

// Adjoint gradient, element term: g[e] = - sum_k lambda_k,e^T K_ref u_k,e,
// one thread per element. K_ref[a][b] of the Q1 element depends only on the
// number of coordinate bits in which local nodes a and b differ (coef[0..3]);
// Dirichlet nodes carry 0.
template <int DIM>
__global__ void k_elem_grad(int ne, int nrhs, double c0, double c1, double c2, double c3,
                            const double* __restrict__ u, const double* __restrict__ lam, double* __restrict__ g) {
  constexpr int NL = 1 << DIM;
  const int64_t n1 = ne + 1;
  const int64_t n_el = DIM == 2 ? (int64_t)ne * ne : (int64_t)ne * ne * ne;
  const double coef[4] = {c0, c1, c2, c3};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
    const int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = DIM == 3 ? (int)(e / ((int64_t)ne * ne)) : 0;
    int64_t node[NL];
    bool live[NL];
#pragma unroll
    for (int a = 0; a < NL; ++a) {
      const int bx = ex + (a & 1), by = ey + ((a >> 1) & 1), bz = DIM == 3 ? ez + ((a >> 2) & 1) : 0;
      node[a] = bx + n1 * (by + n1 * (int64_t)bz);
      live[a] = !(bx == 0 || bx == ne || by == 0 || by == ne || (DIM == 3 && (bz == 0 || bz == ne)));
    }
    double s = 0.0;
    for (int k = 0; k < nrhs; ++k) {
      double uv[NL], lv[NL];
#pragma unroll
      for (int a = 0; a < NL; ++a) {
        uv[a] = live[a] ? u[node[a] * nrhs + k] : 0.0;
        lv[a] = live[a] ? lam[node[a] * nrhs + k] : 0.0;
      }
#pragma unroll
      for (int a = 0; a < NL; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < NL; ++b) t = fma(coef[__popc(a ^ b)], uv[b], t);
        s = fma(lv[a], t, s);
      }
    }
    g[e] = -s;
  }
}

// ---------------------------------------------------------------------------
// PCG vector kernels
// ---------------------------------------------------------------------------
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

// Interior solves with the sparse local solver: A_II^-1 X for all
// subdomains at once by the forward and backward sweeps of the interior
// forest (X and the result in compact interior order); with yscatter the
// result goes through W.tI to rows yscatter of Y.
cudaError_t interior_sweeps(bddc_handle_s* h, const ApplyWork& W, const double* X, double* Y,
                            const int32_t* yscatter, int nrhs, cudaStream_t st) {
  if (h->nI_tot == 0) return cudaSuccess;
  double* out = yscatter ? W.tI : Y;
  cudaError_t e = launch_sweeps(h, h->is, X, W.ir, W.iy, out, nrhs, st, false, false);
  if (e != cudaSuccess || !yscatter) return e;
  h->launches++;
  return launch_scatter_rows(h->nI_tot, nrhs, yscatter, out, Y, st);
}

// One batched application of the interior (A_II^-1) or interface (K_GG)
// operators of all subdomains.
// Y = Op X over the interior or interface operators; counts its launches.
cudaError_t local_op(bddc_handle_s* h, bool interior, const double* X, double* Y, const int32_t* yscatter, int nrhs,
                     cudaStream_t st, int max_per_sm = 0) {
  if (interior && h->sparse_local) return interior_sweeps(h, h->w, X, Y, yscatter, nrhs, st);
  if (h->use_tc) return launch_tc_gemm(h, interior, X, Y, yscatter, nrhs, st);
  if (h->use_sym) {
    if (nrhs != 1) return cudaErrorInvalidValue;   // nrhs_max is 1 on this path
    h->launches += (interior ? h->n_wsy_I : h->n_wsy_G) > 0;
    return interior ? launch_sgemv_tma(h->precision, h->d_wsy_I, h->n_wsy_I, h->max_n_I, h->d_aii, X, Y, yscatter,
                                       h->d_err, st, h->tune_stage_kb[0], h->tune_sym_stages[0], max_per_sm)
                    : launch_sgemv_tma(h->precision, h->d_wsy_G, h->n_wsy_G, h->max_n_G, h->d_kgg, X, Y, yscatter,
                                       h->d_err, st, h->tune_stage_kb[1], h->tune_sym_stages[1], max_per_sm);
  }
  h->launches += (interior ? h->n_wi_I : h->n_wi_G) > 0;
  if (h->use_tma)
    return interior ? launch_bgemv_tma(h->precision, h->d_wtx_I[h->tune_tile_class[0]],
                                       h->n_wtx_I[h->tune_tile_class[0]], h->max_cols_I, h->d_aii, X, Y, yscatter,
                                       nrhs, h->d_err, st, h->tune_stage_kb[0], max_per_sm)
                    : launch_bgemv_tma(h->precision, h->d_wtx_G[h->tune_tile_class[1]],
                                       h->n_wtx_G[h->tune_tile_class[1]], h->max_cols_G, h->d_kgg, X, Y, yscatter,
                                       nrhs, h->d_err, st, h->tune_stage_kb[1], max_per_sm);
  return interior ? bgemv(h->precision, h->d_wi_I, h->n_wi_I, h->max_cols_I, h->d_aii, X, Y, yscatter, nrhs, st)
                  : bgemv(h->precision, h->d_wi_G, h->n_wi_G, h->max_cols_G, h->d_kgg, X, Y, yscatter, nrhs, st);
}

}  // namespace

// e_G = Phi_G u_c for every interface copy (k_phi_prolong).
cudaError_t launch_phi_prolong(bddc_handle_s* h, const ApplyWork& W, int nrhs, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>(h->n_sub, 16 * 152);
  const bool f32 = h->phi_prec == BDDC_PREC_FP32;
  const size_t smem = (size_t)std::max(1, h->max_nc) * nrhs * (f32 ? 4 : 8);
  cudaError_t e = cudaSuccess;
  if (f32) {
    auto kern = nrhs == 1 ? k_phi_prolong<float, 1> : k_phi_prolong<float, 8>;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    kern<<<blocks, kThreads, smem, st>>>(h->n_sub, nrhs, static_cast<const float*>(h->d_phit), h->d_pt_off,
                                         h->d_pt_ld, h->d_sub_goff, h->d_sub_coff, h->d_ccdof, W.uc, W.eG);
  } else {
    auto kern = nrhs == 1 ? k_phi_prolong<double, 1> : k_phi_prolong<double, 8>;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    kern<<<blocks, kThreads, smem, st>>>(h->n_sub, nrhs, static_cast<const double*>(h->d_phit), h->d_pt_off,
                                         h->d_pt_ld, h->d_sub_goff, h->d_sub_coff, h->d_ccdof, W.uc, W.eG);
  }
  h->launches++;
  return cudaGetLastError();
}

cudaError_t launch_local_op(bddc_handle_s* h, bool interior, const double* X, double* Y, int nrhs, cudaStream_t st) {
  return local_op(h, interior, X, Y, nullptr, nrhs, st);
}

cudaError_t launch_interior_correction(bddc_handle_s* h, const double* b, double* x, int nrhs,
                                       cudaStream_t st) {
  // x = 0 on interface and Dirichlet nodes, A_II^-1 b_I on interior nodes
  k_restrict<false><<<blocks_for(h->nI_tot * nrhs), kThreads, 0, st>>>(b, nrhs, h->d_inode, h->nI_tot, nullptr,
                                                                nullptr, 0, h->w.rI, nullptr, h->d_dnode,
                                                                h->n_dir, x);
  if (h->n_gu)
    k_zero_nodes<<<blocks_for(h->n_gu * nrhs), kThreads, 0, st>>>(h->n_gu, nrhs, h->d_gu_node, x);
  cudaError_t e = local_op(h, true, h->w.rI, x, h->d_inode, nrhs, st);
  h->launches += 1 + (h->n_gu > 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_apply(bddc_handle_s* h, const double* r, double* z, int nrhs, cudaStream_t st,
                         cudaEvent_t* ev, const ApplyWork* wk) {
  const ApplyWork& W = wk ? *wk : h->w;
  cudaError_t e;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], st);
  };
  mark(0);
  // restriction: the compact r_I (W r_G is formed by the interface
  // right-hand side, the Dirichlet rows of z by the prolongation)
  if (h->nI_tot) {
    (nrhs == 1 ? k_restrict<true> : k_restrict<false>)<<<blocks_for(h->nI_tot * nrhs), kThreads, 0, st>>>(
        r, nrhs, h->d_inode, h->nI_tot, nullptr, nullptr, 0, W.rI, nullptr, nullptr, 0, nullptr);
    h->launches++;
  }
  mark(1);
  // t_I = A_II^-1 r_I
  if ((e = local_op(h, true, W.rI, W.tI, nullptr, nrhs, st)) != cudaSuccess) return e;
  mark(2);
  if (h->nG_tot) {
    // y'_G = W r_G - A_GI t_I; z_G = K_GG y'_G
    (nrhs == 1 ? k_iface_rhs<1, true> : k_iface_rhs<1, false>)<<<blocks_for(h->nG_tot * nrhs), kThreads, 0, st>>>(
        h->nG_tot, nrhs, h->d_agi_ptr, h->d_agi_col, h->d_agi_val, W.tI, h->d_gnode, h->d_gw, r, W.yG);
    h->launches++;
  }
  mark(3);
  // The interface operator (z_G = K_GG y'_G) and the coarse residual and
  // solve depend only on y'_G: with tune_overlap they run concurrently, the
  // interface operator on a second stream capped at `cap` blocks per SM, the
  // coarse sweeps on one block of 256 (one column) or 512 threads per SM, so
  // that both fit on every SM at once (the coarse kernel is cooperative: its
  // grid must be resident). Registers decide the cap: a symmetric-GEMV block
  // holds 288 x 72 and a 256-thread sweep block 256 x 128 of the SM's 65536,
  // so one of the former fits beside the latter; a streamed-GEMV block
  // (288 x 56) fits twice.
  const int ax = h->aux_sel;
  const bool overlap = h->tune_overlap && h->nG_tot && h->n_c && !h->coarse_dense && h->aux_stream[ax];
  const int cap = h->use_sym ? 1 : 2;
  if (overlap) {
    if ((e = cudaEventRecord(h->ev_fork[ax], st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->aux_stream[ax], h->ev_fork[ax], 0)) != cudaSuccess) return e;
    if ((e = local_op(h, false, W.yG, W.zG, nullptr, nrhs, h->aux_stream[ax], cap)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(h->ev_join[ax], h->aux_stream[ax])) != cudaSuccess) return e;
  } else if (h->nG_tot) {
    if ((e = local_op(h, false, W.yG, W.zG, nullptr, nrhs, st)) != cudaSuccess) return e;
  }
  mark(4);
  if (h->n_c) {
    // coarse residual r_c = sum R_ci^T Phi_G^T y'_G
    if ((e = launch_bgemv_tma(h->phi_prec, h->d_wi_PT, h->n_wi_PT, h->max_ld_PT, h->d_phit, W.yG, W.g,
                              nullptr, nrhs, h->d_err, st, 12, overlap ? cap : 0)) != cudaSuccess)
      return e;
    (nrhs == 1 ? k_coarse_gather<true> : k_coarse_gather<false>)<<<blocks_for(h->n_c * nrhs), kThreads, 0, st>>>(
        h->n_c, nrhs, h->d_cg_ptr, h->d_cg_idx, W.g, W.rc);
    h->launches += 2;
  }
  mark(5);
  if (h->n_c) {
    if (h->coarse_dense) {
      // u_c = A_c^-1 r_c: per-panel products of the explicit inverse, then their sum
      if ((e = launch_bgemv_tma(BDDC_PREC_FP64, h->d_wi_C, h->n_wi_C, h->ldc, h->d_acinv, W.rc, W.cpart,
                                nullptr, nrhs, h->d_err, st)) != cudaSuccess)
        return e;
      k_panel_sum<<<blocks_for(h->n_c * nrhs), kThreads, 0, st>>>(h->n_c * nrhs, h->n_cpanels, W.cpart,
                                                                  W.uc);
      h->launches += 2;
    } else {
      // u_c = A_c^-1 r_c: sparse Cholesky forward and backward sweeps
      if ((e = launch_coarse_solve(h, W, W.rc, W.uc, nrhs, st, overlap)) != cudaSuccess) return e;
    }
  }
  if (overlap && (e = cudaStreamWaitEvent(st, h->ev_join[ax], 0)) != cudaSuccess) return e;
  mark(6);
  if (h->n_gu) {
    // v_G = sum R^T W (z_G + Phi_G u_c)
    const double* eG = nullptr;
    if (h->n_c) {
      if ((e = launch_phi_prolong(h, W, nrhs, st)) != cudaSuccess) return e;
      eG = W.eG;
    } else {
      cudaMemsetAsync(W.eG, 0, sizeof(double) * h->nG_tot * nrhs, st);
      eG = W.eG;
    }
    (nrhs == 1 ? k_prolong_gather<1, true> : k_prolong_gather<1, false>)<<<
        blocks_for(std::max(h->n_gu, h->n_dir) * nrhs), kThreads, 0, st>>>(
        h->n_gu, nrhs, h->d_gu_node, h->d_gu_ptr, h->d_gu_copy, h->d_gw, W.zG, eG, z, h->d_dnode, h->n_dir);
    h->launches++;
  } else if (h->n_dir) {
    k_zero_nodes<<<blocks_for(h->n_dir * nrhs), kThreads, 0, st>>>(h->n_dir, nrhs, h->d_dnode, z);
    h->launches++;
  }
  mark(7);
  // z_I = A_II^-1 (r_I - A_IG v_G)
  if (h->nI_tot) {
    (nrhs == 1 ? k_interior_rhs<1, true> : k_interior_rhs<1, false>)<<<blocks_for(h->nI_tot * nrhs), kThreads, 0,
                                                                        st>>>(
        h->nI_tot, nrhs, h->d_aig_ptr, h->d_aig_col, h->d_aig_val, h->d_inode, r, z, W.bI);
    h->launches++;
  }
  mark(8);
  if ((e = local_op(h, true, W.bI, z, h->d_inode, nrhs, st)) != cudaSuccess) return e;
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

cudaError_t launch_gather_rows(int64_t n, int nrhs, const int32_t* perm, const double* src, double* dst,
                               cudaStream_t st) {
  if (n * nrhs == 0) return cudaSuccess;
  k_gather_rows<<<blocks_for(n * nrhs), kThreads, 0, st>>>(n, nrhs, perm, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_scatter_rows(int64_t n, int nrhs, const int32_t* perm, const double* src, double* dst,
                                cudaStream_t st) {
  if (n * nrhs == 0) return cudaSuccess;
  (nrhs == 1 ? k_scatter_rows<true> : k_scatter_rows<false>)<<<blocks_for(n * nrhs), kThreads, 0, st>>>(
      n, nrhs, perm, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_elem_grad(bddc_handle_s* h, const double* u, const double* lam, double* g, int nrhs,
                             cudaStream_t st) {
  double c[4];
  q1_coefs(h->dim, h->h, false, c);   // K_ref: the stiffness coefficients for sigma = 1
  if (h->dim == 2)
    k_elem_grad<2><<<blocks_for(h->n_elems), kThreads, 0, st>>>(h->ne, nrhs, c[0], c[1], c[2], c[3], u, lam, g);
  else
    k_elem_grad<3><<<blocks_for(h->n_elems), kThreads, 0, st>>>(h->ne, nrhs, c[0], c[1], c[2], c[3], u, lam, g);
  h->launches++;
  return cudaGetLastError();
}




cudaError_t launch_update_p(bddc_handle_s* h, int nrhs, cudaStream_t st) {
  k_update_p<<<blocks_for(h->n_nodes * nrhs), kThreads, 0, st>>>(h->n_nodes, nrhs, h->d_scal + S_BETA * h->nrhs_max,
                                                                 h->p_z, h->p_p, h->p_zold);
  h->launches++;
  return cudaGetLastError();
}

namespace {
__global__ void k_loop_control(int32_t* gflags, int maxit, int first, cudaGraphConditionalHandle cond) {
  const int it = first ? 1 : gflags[3] + 1;
  gflags[3] = it;
  cudaGraphSetConditional(cond, (gflags[0] > 0 && it < maxit && gflags[2] == 0) ? 1u : 0u);
}
}  // namespace

cudaError_t launch_loop_control(bddc_handle_s* h, int maxit, int first, cudaGraphConditionalHandle cond,
                                cudaStream_t st) {
  k_loop_control<<<1, 1, 0, st>>>(h->d_iscal + I_COUNT * h->nrhs_max, maxit, first, cond);
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
