// Launch wrappers for the libbddc device kernels (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.hpp"

namespace bddc {

// z = M^-1 r for nrhs columns; all phases on `st`. prof_events, if not
// null, holds 10 events recorded between the launches.
// W: the work vectors to use (null: the handle's own).
cudaError_t launch_apply(bddc_handle_s* h, const double* r, double* z, int nrhs, cudaStream_t st,
                         cudaEvent_t* prof_events = nullptr, const ApplyWork* W = nullptr);

// Batched GEMV over row tiles of many operators, streamed by bulk async
// copies through shared memory (bddc_bgemv_tma.cu). err receives
// BDDC_ERR_TIMEOUT if a bounded wait runs out.
bool bgemv_tma_supported(int precision, int max_lda);
// Symmetric operators as their packed lower triangle (diagonal halved, rows
// padded to 16 bytes): elements of one n x n operator, whether the streamed
// symmetric GEMV supports the precision (FP32, BF16) and size, and
// Y = Op X for one right-hand side (one work item per operator: moff,
// ncols = n, xoff, yoff).
int64_t sym_packed_elems(int precision, int n);
bool sgemv_tma_supported(int precision, int max_n);
cudaError_t launch_sgemv_tma(int precision, const WorkItem* items, int n_items, int max_n, const void* arena,
                             const double* X, double* Y, const int32_t* yscatter, int32_t* err, cudaStream_t st,
                             int stage_kb, int n_stages, int max_per_sm = 0);
// stage_kb: target bytes of one shared-memory stage, in KB (1..64; 12 by default,
// the autotuner may choose another per operator family); max_per_sm > 0 caps
// the blocks per SM (to leave room for a concurrent kernel).
cudaError_t launch_bgemv_tma(int precision, const WorkItem* items, int n_items, int max_lda, const void* arena,
                             const double* X, double* Y, const int32_t* yscatter, int nrhs, int32_t* err,
                             cudaStream_t st, int stage_kb = 12, int max_per_sm = 0);

// Tensor-core batched GEMM for blocks of right-hand sides (bddc_tc_gemm.cu).
// Host packing of dense n x n operators (row-major float64) into the tiled
// layout; per operator opinfo holds {xoff, n, first packed column, first
// 16-byte column slice}, slice_op maps every 16-byte column slice of the
// packed operand to its operator.
template <typename T> struct TcCvt;
template <> struct TcCvt<float> {
  static float from(double v) { return (float)v; }
};
template <> struct TcCvt<__nv_bfloat16> {
  static __nv_bfloat16 from(double v) { return __float2bfloat16_rn((float)v); }
};
template <typename T> struct TcPacked {
  std::vector<T> arena;
  std::vector<TcUnit> units;
  std::vector<int32_t> slice_op;
  std::vector<int32_t> opinfo;
  int64_t cols_total = 0;
  int max_g = 0;   // most row tiles in one unit
};
template <typename T>
void tc_pack_host(const std::vector<std::vector<double>>& ops, const std::vector<int>& dims,
                  const std::vector<int32_t>& xoff, TcPacked<T>& out);
// Bytes of the packed operand buffer for operators of cols_total padded columns.
size_t tc_operand_bytes(int precision, int64_t cols_total, int nrhs_max);
// Y = Op X over the interior (A_II^-1) or interface (K_GG) operators;
// precision BDDC_PREC_BF16 (kind::f16) or BDDC_PREC_TF32 (kind::tf32).
cudaError_t launch_tc_gemm(bddc_handle_s* h, bool interior, const double* X, double* Y, const int32_t* yscatter,
                           int nrhs, cudaStream_t st);

// dst[i, k] = src[perm[i], k] for i < n, k < nrhs (row gather).
cudaError_t launch_gather_rows(int64_t n, int nrhs, const int32_t* perm, const double* src, double* dst,
                               cudaStream_t st);

// dst[perm[i], k] = src[i, k] for i < n, k < nrhs (row scatter).
cudaError_t launch_scatter_rows(int64_t n, int nrhs, const int32_t* perm, const double* src, double* dst,
                                cudaStream_t st);

// Sweeps of a supernodal factorisation (coarse_solve.cu). build_sweeps
// uploads cf (dofs numbered in elimination order or not) into S: the gather
// form for one right-hand side on a grid of blocks_req blocks (0 = one per
// SM), and with `multi` also the node matrices and unit lists for several.
// form: kSweepCoop (one cooperative launch of the gather form: small
// factors), kSweepLevel (gather form, one launch per phase, sub-warp groups
// sized to the rows) or kSweepBlock (supernode by supernode with the dense
// node matrices streamed, one launch per phase; the level form where a front
// does not fit in shared memory). coef32: the one-column form's coefficients
// in float32 (products and sums in float32; the per-level form only).
cudaError_t build_sweeps(bddc_handle_s* h, const CoarseFactor& cf, SweepSet& S, bool multi, int blocks_req,
                         int form, bool coef32);
// u = A^-1 r by the forward and backward sweeps of S, level by level, in one
// cooperative launch (r and u: S.n x nrhs in dof order; rp and y: work
// vectors of the same size). inject: the barriers take the handle's test
// settings (bddc_test_coarse_stall); otherwise the normal limit.
cudaError_t launch_sweeps(bddc_handle_s* h, const SweepSet& S, const double* r, double* rp, double* y, double* u,
                          int nrhs, cudaStream_t st, bool narrow, bool inject);
// Sparse coarse solve: upload of the factorisation of A_c into the handle's
// coarse sweep set; u_c = A_c^-1 r_c by its sweeps.
cudaError_t build_coarse_device(bddc_handle_s* h, const CoarseFactor& cf);
// Inexact coarse solve by plain CG (A_c uploaded by the caller): barrier
// counter and launch checks.
cudaError_t build_coarse_cg_device(bddc_handle_s* h);
// narrow: one block per SM sized to leave room on every SM for a concurrent
// kernel (the interface operator) while the sweeps run: 256 threads (half
// the registers) for one column, 512 threads for several.
cudaError_t launch_coarse_solve(bddc_handle_s* h, const ApplyWork& W, const double* rc, double* uc, int nrhs,
                                cudaStream_t st, bool narrow = false);

// Y = Op X over the interior (A_II^-1) or interface (K_GG) operators in the
// compact layouts, on whichever engine the handle uses (for the autotuner).
cudaError_t launch_local_op(bddc_handle_s* h, bool interior, const double* X, double* Y, int nrhs, cudaStream_t st);

// x = P_I b: interior correction of b (zero on interface and Dirichlet nodes).
cudaError_t launch_interior_correction(bddc_handle_s* h, const double* b, double* x, int nrhs,
                                       cudaStream_t st);

// b = (M f) on the free nodes (matrix-free Q1 mass matrix).
cudaError_t launch_rhs(bddc_handle_s* h, const double* f, double* b, int nrhs, cudaStream_t st);

// g[e] = - sum_k lambda_k,e^T K_ref u_k,e (adjoint gradient, element term).
cudaError_t launch_elem_grad(bddc_handle_s* h, const double* u, const double* lam, double* g, int nrhs,
                             cudaStream_t st);

// PCG scalar updates applied by the last block of a reducing kernel.
enum FinalizeOp { FIN_INIT = 0, FIN_RHO = 1, FIN_ALPHA = 2, FIN_CONV = 3, FIN_BETA = 4 };

// Global SpMV (bddc_pcg.cu): coefficients of the assembled Q1 stencil
// (the centre and the forward half of the symmetric couplings, each array
// with zero guard zones of stencil_guard entries on both sides), built once
// per handle; y = A x, and with op >= 0 also x.y per column followed by the
// PCG scalar update `op`.
int stencil_points(int dim);
int64_t stencil_guard(int dim, int ne);
cudaError_t launch_build_stencil(bddc_handle_s* h, cudaStream_t st);
cudaError_t launch_spmv(bddc_handle_s* h, const double* x, double* y, int nrhs, int op, double rtol, int flexible,
                        cudaStream_t st);
// x += alpha p; r -= alpha q; r.r; stop test.
cudaError_t launch_update_xr_conv(bddc_handle_s* h, double* x, int nrhs, double rtol, int flexible,
                                  cudaStream_t st);
// a0.b0 (and a1.b1) per column, then the PCG scalar update `op`.
cudaError_t launch_dots_fin(bddc_handle_s* h, int nrhs, const double* a0, const double* b0, const double* a1,
                            const double* b1, int op, double rtol, int flexible, cudaStream_t st);

// p = z + beta p; zold = z.
cudaError_t launch_update_p(bddc_handle_s* h, int nrhs, cudaStream_t st);
// r = b - q; p = 0; zold = 0 (start of PCG, q = A x0).
cudaError_t launch_residual(bddc_handle_s* h, const double* b, int nrhs, cudaStream_t st);

// Offsets of the per-column PCG scalars inside h->d_scal (times nrhs_max).
enum ScalarSlot { S_RHO = 0, S_ALPHA, S_BETA, S_BB, S_RR, S_RELRES, S_COUNT };
enum IntSlot { I_ACTIVE = 0, I_ITERS, I_STATUS, I_COUNT };
// global int flags after the per-column ones: [0] active columns, [1] breakdown,
// [2] device error (BDDC_ERR_TIMEOUT from a bounded wait), sticky until setup,
// [3] iterations done by the whole-solve graph
constexpr int kGlobalFlags = 4;

// Loop control of the whole-solve graph (after the first iteration with
// first = 1, then after every iteration of the conditional body): counts the
// iteration and sets the WHILE condition to (an active column, fewer than
// maxit iterations, no device wait ran out).
cudaError_t launch_loop_control(bddc_handle_s* h, int maxit, int first, cudaGraphConditionalHandle cond,
                                cudaStream_t st);
constexpr int kRedBlocks = 1216;  // 8 x 152 SMs: blocks (and fixed-order partials) of the reducing kernels

}  // namespace bddc
