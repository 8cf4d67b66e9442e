// Launch wrappers for the libbddc device kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"

namespace bddc {

// z = M^-1 r for nrhs columns; all phases on `st`. prof_events, if not
// null, holds 10 events recorded between the launches.
cudaError_t launch_apply(bddc_handle_s* h, const double* r, double* z, int nrhs, cudaStream_t st,
                         cudaEvent_t* prof_events = nullptr);

// x = P_I b: interior correction of b (zero on interface and Dirichlet nodes).
cudaError_t launch_interior_correction(bddc_handle_s* h, const double* b, double* x, int nrhs,
                                       cudaStream_t st);

// y = A x (matrix-free Q1 stiffness on the free nodes).
cudaError_t launch_matvec(bddc_handle_s* h, const double* x, double* y, int nrhs, cudaStream_t st);

// b = (M f) on the free nodes.
cudaError_t launch_rhs(bddc_handle_s* h, const double* f, double* b, int nrhs, cudaStream_t st);

// Partial per-column sums of up to three elementwise products over all
// nodes, into h->d_partials[block][slot][k].
cudaError_t launch_dots(bddc_handle_s* h, int nrhs, const double* a0, const double* b0,
                        const double* a1, const double* b1, const double* a2, const double* b2,
                        cudaStream_t st);

// PCG scalar updates (one block; fixed summation order over the partials).
enum FinalizeOp { FIN_INIT = 0, FIN_RHO = 1, FIN_ALPHA = 2, FIN_CONV = 3, FIN_BETA = 4 };
cudaError_t launch_finalize(bddc_handle_s* h, int op, int nrhs, double rtol, int flexible,
                            cudaStream_t st);

// x += alpha p; r -= alpha q (per-column alpha on the device).
cudaError_t launch_update_xr(bddc_handle_s* h, double* x, int nrhs, cudaStream_t st);
// p = z + beta p; zold = z.
cudaError_t launch_update_p(bddc_handle_s* h, int nrhs, cudaStream_t st);
// r = b - q (initial residual, q = A x0).
cudaError_t launch_residual(bddc_handle_s* h, const double* b, int nrhs, cudaStream_t st);

// Offsets of the per-column PCG scalars inside h->d_scal (times nrhs_max).
enum ScalarSlot { S_RHO = 0, S_ALPHA, S_BETA, S_BB, S_RR, S_RELRES, S_COUNT };
enum IntSlot { I_ACTIVE = 0, I_ITERS, I_STATUS, I_COUNT };
// global int flags after the per-column ones: [0] active columns, [1] breakdown
constexpr int kRedBlocks = 304;   // 2 x 152 SMs for the dot-product partials

}  // namespace bddc
