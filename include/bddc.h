/*
 * bddc.h — C ABI of libbddc: BDDC-preconditioned conjugate gradients for Q1
 * finite-element diffusion problems on a subdomain decomposition, on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Goebel, Cojean, Anzt, "BDDC preconditioning on GPUs for Cardiac
 * Simulations" (arXiv 2410.14786), Sec. 2:
 *   A = sum_i R_i^T A_i R_i                          (subassembly)
 *   [A_i C_i^T; C_i 0][Phi_i; Lambda_i] = [0; I]      (Eq. saddlepoint)
 *   A_c = sum_i R_ci^T Phi_i^T A_i Phi_i R_ci
 *   r_c = sum_i R_ci^T Phi_i^T W_i R_i r
 *   v1  = sum_i R_i^T W_i Phi_i R_ci A_c^-1 r_c        (Eq. coarsegrid)
 *   [A_i C_i^T; C_i 0][z_i; lambda_i] = [W_i R_i r; 0] (Eq. compzi)
 *   v2  = sum_i R_i^T W_i z_i                          (Eq. localsubdomain)
 *   r1  = r - A (v1 + v2)
 *   v3  = sum_i R_i^T R_Ii^T (R_Ii A_i R_Ii^T)^-1 R_Ii R_i r1   (Eq. inner)
 *   M^-1 r = v1 + v2 + v3
 * with corner values and edge / face averages as constraints C_i and weights
 * W_i = diag(1 / kappa), kappa = number of subdomains sharing a dof (Sec. 2).
 *
 * Problem: -div(sigma grad u) = f on the unit square (dim 2) or cube (dim 3),
 * ne elements per direction, Q1 elements, one conductivity per element,
 * homogeneous Dirichlet conditions on the whole boundary (those nodes are
 * eliminated). The library takes the problem unassembled (elements and
 * their subdomain ids), because the local Neumann matrices A_i cannot be
 * recovered from an assembled A.
 *
 * Numbering: node (ix, iy[, iz]) is ix + (ne+1) * (iy + (ne+1) * iz);
 * element (ex, ey[, ez]) is ex + ne * (ey + ne * ez).
 *
 * Vectors: every vector argument is an array of n_nodes * nrhs doubles,
 * node-major with the right-hand side index fastest (entry (node, k) at
 * node * nrhs + k). Entries at Dirichlet nodes are ignored on input and
 * written as 0 on output. Unless stated otherwise vectors are DEVICE
 * pointers owned by the caller; they must not alias each other.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream). Calls on one handle are not re-entrant: do not run two
 * calls on the same handle concurrently, on any streams or host threads.
 * Devices: a call makes the handle's device current while it runs and
 * restores the caller's current device before it returns.
 *
 * Errors: every int-returning call returns BDDC_OK (0) on success, a
 * negative BDDC_ERR_* code on failure, or BDDC_NOT_CONVERGED (positive) from
 * bddc_pcg_solve. bddc_strerror() gives a message; bddc_last_error() gives
 * the detail of the most recent failure on the calling thread.
 */
#ifndef BDDC_H
#define BDDC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BDDC_OK               0
#define BDDC_NOT_CONVERGED    1   /* maxit reached before rtol (solve only) */
#define BDDC_ERR_INVALID_ARG (-1) /* bad argument: sizes, ids, sigma <= 0, NaN */
#define BDDC_ERR_OOM         (-2) /* device or host allocation failed */
#define BDDC_ERR_CUDA        (-3) /* a CUDA runtime call failed */
#define BDDC_ERR_SINGULAR    (-4) /* non-positive pivot in a setup factorisation */
#define BDDC_ERR_TIMEOUT     (-5) /* a bounded device wait ran out */
#define BDDC_ERR_BREAKDOWN   (-6) /* PCG breakdown: p^T A p <= 0 or non-finite */
#define BDDC_ERR_NO_DEVICE   (-7) /* no CUDA device, or not an sm_103 device */

/* ---- options ---------------------------------------------------------- */
/* Precision of the batched local and interior operators (the explicit
 * local constrained-Neumann and interior-Dirichlet operators). The outer
 * PCG vectors, dot products, SpMV, setup factorisations and the coarse
 * factorisation and solve are float64 in every mode. The coarse basis
 * Phi_i (coarse residual Phi_i^T y_i and prolongation Phi_i u_c) is float64
 * in the FP64 mode, and float32 with float32 accumulation in the FP32,
 * BF16 and TF32 modes unless bddc_options_t.phi_fp64 is set. FP64 runs standard
 * PCG; the other modes run flexible PCG. */
#define BDDC_PREC_FP64  0
#define BDDC_PREC_FP32  1   /* float32 operators, float32 accumulation */
#define BDDC_PREC_BF16  2   /* bfloat16 operators, float32 accumulation */
#define BDDC_PREC_TF32  3   /* float32 operators read as TF32 by the tensor cores
                               (tcgen05 kind::tf32), float32 accumulation */

/* Where the local and interior operators run. AUTO: tensor cores (tcgen05,
 * operators stored in the MMA tile layout) for BF16 and TF32 when nrhs_max
 * >= 8, the streamed CUDA-core GEMV otherwise; below 8 right-hand sides a
 * TF32 request runs the FP32 form (float32 operators on the CUDA cores, as
 * BDDC_PREC_FP32), because an MMA of N = 16 would waste most of its work:
 * bddc_info_t.precision then reports BDDC_PREC_FP32. ON: tensor cores for
 * BF16 and TF32 whatever nrhs_max. OFF: CUDA cores (invalid with TF32).
 * On the tensor cores the float64 operand is split into a high and a low
 * part in the operator's format (two MMAs per K step), so only the operator
 * carries the form's rounding. */
#define BDDC_TC_AUTO 0
#define BDDC_TC_ON   1
#define BDDC_TC_OFF  2

/* Coarse solve (float64). DENSE: the explicit inverse of A_c, applied as
 * one matrix-vector product (n_c^2 float64 multiply-adds). SPARSE: a
 * nested-dissection supernodal Cholesky factorisation applied by
 * level-scheduled sweeps (far fewer operations and bytes; needed when the
 * dense inverse does not fit). AUTO = SPARSE. Both are exact. CG: the
 * paper's choice (Sec. 3: the coarse system of Eq. coarsegrid solved with
 * plain CG): unpreconditioned conjugate gradients on A_c from u_c = 0, every
 * column until ||r_k|| <= coarse_cg_rtol ||r_c|| or coarse_cg_maxit
 * iterations, in one cooperative launch; no coarse factorisation at setup.
 * The preconditioner is then inexact (it varies with r), so bddc_pcg_solve
 * runs flexible PCG in every precision. */
#define BDDC_COARSE_AUTO    0
#define BDDC_COARSE_DENSE   1
#define BDDC_COARSE_SPARSE  2
#define BDDC_COARSE_CG      3

/* Local solver of the interior (Dirichlet) problems with A_II (Sec. 2, Eqs.
 * compzi and inner; Sec. 3, implementation paragraph: the paper factorises
 * its local systems with a sparse direct solver on the GPU). DENSE: A_II^-1
 * is formed explicitly in float64 and stored in the operator precision;
 * every interior solve is a dense product with it. SPARSE: A_II is
 * factorised by a supernodal Cholesky factorisation in nested-dissection
 * order of the subdomain's elements, in float64, and every interior solve
 * is the factor's forward and backward sweeps, level by level (float64 in
 * every precision); the interface Schur complement comes from the same
 * factorisation, so no dense n_I x n_I matrix is formed at any point (for
 * subdomains of 10^4 dofs and more, as in the experiments of Sec. 3, whose
 * dense A_II^-1 would take gigabytes each). K_GG is dense in both. */
#define BDDC_LOCAL_DENSE    0
#define BDDC_LOCAL_SPARSE   1

/* Constraint families that become coarse (primal) dofs (Sec. 2). */
#define BDDC_CORNERS 1u
#define BDDC_EDGES   2u
#define BDDC_FACES   4u

typedef struct bddc_handle_s *bddc_handle_t;

typedef struct {
    int32_t dim;                    /* 2 or 3 */
    int32_t ne;                     /* elements per direction, >= 1 */
    const double *elem_sigma;       /* [ne^dim] HOST, finite, > 0 */
    const int32_t *elem_subdomain;  /* [ne^dim] HOST, each in [0, n_sub) */
    int32_t n_sub;                  /* number of subdomains, each non-empty */
} bddc_problem_t;

typedef struct {
    int32_t precision;     /* BDDC_PREC_* */
    uint32_t constraints;  /* BDDC_CORNERS | BDDC_EDGES | BDDC_FACES; 0 = all */
    int32_t nrhs_max;      /* largest nrhs any later call uses, 1..64 */
    int32_t n_threads;     /* host threads for setup; 0 = all cores */
    int32_t device;        /* CUDA device ordinal */
    int32_t coarse;        /* BDDC_COARSE_* */
    int32_t no_graph;      /* 1: launch every PCG iteration's kernels directly instead of
                              replaying a captured CUDA graph (for profilers) */
    int32_t phi_fp64;      /* 1: keep Phi_i in float64 in the FP32, BF16 and TF32 modes too */
    int32_t tensor_cores;  /* BDDC_TC_* */
    int32_t coarse_blocks; /* blocks of the one-column sparse coarse solve (one per SM at
                              most); 0 = one per SM. Fewer blocks give each warp more
                              units of every level (for small coarse problems). >= 0 */
    int32_t full_operators; /* 1: store the symmetric local operators in full. 0 (default):
                              in the FP32 and BF16 forms on the CUDA cores with
                              nrhs_max = 1, A_II^-1 and K_GG are stored as their lower
                              triangles (about half the bytes) and applied by the
                              symmetric streamed GEMV; elsewhere in full */
    int32_t history;       /* PCG iterations whose scalars (||r_k||, alpha_k, beta_k) the
                              handle keeps for bddc_pcg_history, 0..100000; 0 = none */
    int32_t coarse_cg_maxit; /* BDDC_COARSE_CG: iteration limit of the coarse CG, >= 0;
                              0 = 2000 */
    double coarse_cg_rtol; /* BDDC_COARSE_CG: relative residual at which the coarse CG
                              stops, in [0, 1); 0 = 1e-10 */
    int32_t local_solver;  /* BDDC_LOCAL_*; 0 = DENSE */
    int32_t local_leaf;    /* BDDC_LOCAL_SPARSE: largest vertex set of the nested dissection
                              that is not split further (a dense front), 0..4096; 0 = 32 */
} bddc_options_t;

typedef struct {
    int64_t n_nodes, n_free, n_interior, n_interface_nodes;
    int64_t n_sub, n_c;                 /* subdomains, coarse dofs (globs) */
    int64_t n_corners, n_edges, n_faces;
    int64_t sum_ni, sum_nI2, sum_nG2;   /* sum n_i, sum n_I^2, sum n_Gamma^2 */
    int64_t sum_nG_nc;                  /* sum n_Gamma * n_ci */
    int64_t max_ni;
    int64_t operator_bytes;             /* device bytes of the local / interior operators */
    int64_t coarse_bytes;               /* device bytes of the coarse operator */
    int64_t device_bytes;               /* all device memory the handle holds */
    int64_t apply_bytes_1rhs;           /* algorithmic HBM bytes of one apply, nrhs = 1 */
    int64_t interior_op_bytes;          /* bytes of all A_II^-1 blocks as stored */
    int64_t interface_op_bytes;         /* bytes of all K_GG blocks as stored */
    int64_t n_interface_copies;         /* sum over subdomains of interface nodes */
    int64_t kernel_launches;            /* kernels launched by this handle so far */
    int64_t coarse_factor_entries;      /* stored entries of the coarse operator (dense inverse
                                           or the sparse factor's sweep matrices) */
    int64_t coarse_update_total;        /* sum of the coarse supernodes' update-set sizes */
    int64_t coarse_levels;              /* levels of the coarse elimination tree (0: dense) */
    double setup_seconds;               /* wall time of bddc_setup */
    int32_t precision;                  /* the precision the operators run in (BDDC_PREC_*; see
                                           BDDC_TC_AUTO for TF32 at few right-hand sides) */
    int32_t error_subdomain;            /* subdomain of the last SINGULAR error, else -1 */
    int32_t device_error;               /* BDDC_ERR_TIMEOUT if a bounded device wait of an
                                           earlier call ran out, else 0 (bddc_query synchronises) */
    int32_t phi_precision;              /* BDDC_PREC_FP64 or BDDC_PREC_FP32: storage of Phi_i */
    int32_t tensor_cores;               /* 1 if the local operators run on the tensor cores */
    int32_t solve_graph;                /* 1 if bddc_pcg_solve runs the whole solve as one CUDA graph
                                           (a conditional WHILE node over the iteration), 0 if it
                                           replays one captured iteration at a time or launches
                                           directly */
    int32_t symmetric_operators;        /* 1 if A_II^-1 and K_GG are stored as lower triangles */
    int32_t coarse_cg_iters;            /* BDDC_COARSE_CG: most coarse CG iterations over the columns
                                           of the most recent coarse solve (bddc_query synchronises);
                                           0 otherwise */
    int32_t local_solver;               /* BDDC_LOCAL_* */
    int32_t interior_levels;            /* BDDC_LOCAL_SPARSE: levels of the interior elimination
                                           forest (all subdomains' trees, merged by height); else 0 */
    int64_t interior_factor_entries;    /* BDDC_LOCAL_SPARSE: stored entries of one sweep of the
                                           interior factors (sum over supernodes of (p + u) p);
                                           else 0 */
} bddc_info_t;

/* Build the preconditioner (Sec. 2: the subdomain matrices A_i of A = sum
 * R_i^T A_i R_i, the weights W_i, the corner / edge / face constraints C_i,
 * the coarse basis Phi_i from Eq. saddlepoint, A_c = sum R_ci^T Phi_i^T A_i
 * Phi_i R_ci and its factorisation, and the operators of the local solves
 * of Eqs. compzi and inner; all factorisations in float64 on the host,
 * operators uploaded once to the device). Copies what it needs from
 * `problem`; the caller keeps ownership of every input. On success *out
 * holds a new handle (free it with bddc_destroy); on failure *out is NULL.
 * Errors: INVALID_ARG, SINGULAR (bddc_last_error() names the subdomain),
 * OOM, CUDA, NO_DEVICE. */
int bddc_setup(const bddc_problem_t *problem, const bddc_options_t *options,
               bddc_handle_t *out);

/* z = M^-1 r (Sec. 2: v1 + v2 + v3) for nrhs columns, 1 <= nrhs <=
 * nrhs_max. r and z are device vectors. Asynchronous on `stream`; allocates
 * nothing. */
int bddc_apply(bddc_handle_t h, const double *r, double *z, int32_t nrhs, void *stream);

/* The same z = M^-1 r as bddc_apply, with the apply's temporary vectors in a
 * fixed 8 MiB array that the library reserves on every GPU it is loaded on
 * (held until the process exits), instead of in the handle's workspace. The
 * paper has no counterpart: this is for callers that cannot have device
 * memory allocated on their behalf, for example a host program whose own
 * allocator owns the whole device and forbids cudaMalloc / cudaFree from
 * libraries, or a program that fixes all device memory at start-up. The call
 * itself never calls cudaMalloc, cudaFree or any allocating routine. What
 * moves to the array are the vectors one apply writes and reads (compact
 * interior, interface-copy, constraint and coarse vectors); the handle's
 * other device buffers, allocated once by bddc_setup, are still used: the
 * packed tensor-core operand, the coarse solve's barrier counter and the
 * device error flag.
 * Limit: the temporaries of one apply, (3 n_interior + 3 n_interface_copies
 * + sum n_ci + 2 n_c + C) * nrhs doubles, with C = ceil(n_c / 512) n_c for
 * the dense coarse solve and 2 n_c for the sparse one
 * (sizes from bddc_query; each term rounded up to 32), must not exceed 2^20;
 * larger problems get BDDC_ERR_INVALID_ARG, and so do handles set up with
 * BDDC_COARSE_CG or BDDC_LOCAL_SPARSE (their work vectors are not relocated). The driver places the array in
 * the device's memory when it loads the library's device code on that device:
 * under CUDA's default lazy module loading that happens in the first call on
 * the device (8 MiB less free memory from then on), with
 * CUDA_MODULE_LOADING=EAGER when the context is created. The first call on a
 * device also looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and keeps
 * it for the life of the process; make that first call before any stream
 * capture, and do not use this entry point after cudaDeviceReset or any
 * other teardown of the device's primary context. Every call on every handle of
 * a device shares the one array, and no part of it needs to start at zero
 * (each call writes every element it reads before reading it): calls that
 * overlap on the GPU, on any streams, race and give wrong results. The call
 * does not modify the handle; as for every call on a handle, no other host
 * thread may use the same handle meanwhile. */
int bddc_apply_static_scratch(bddc_handle_t h, const double *r, double *z, int32_t nrhs,
                              void *stream);

/* y = A x (Sec. 2: the global stiffness matrix A = sum R_i^T A_i R_i of
 * the Q1 discretisation on the free nodes, the matrix of the CG iteration of
 * Sec. 3; Dirichlet entries of y are written 0). Device vectors;
 * asynchronous on `stream`. */
int bddc_matvec(bddc_handle_t h, const double *x, double *y, int32_t nrhs, void *stream);

/* b = M f restricted to the free nodes: the load vector of the nodal values
 * f (Q1 interpolant, consistent mass matrix). f holds values at ALL nodes
 * (Dirichlet ones included). Device vectors; asynchronous on `stream`. */
int bddc_rhs(bddc_handle_t h, const double *f, double *b, int32_t nrhs, void *stream);

/* Launch parameters of one handle. The defaults work everywhere;
 * bddc_autotune measures the candidates on the handle's own operators and
 * keeps the fastest. A caller may store the result (e.g. in a file keyed by
 * the problem) and restore it with bddc_set_tuning. */
typedef struct {
    int32_t gemv_stage_kb_interior;   /* streamed-GEMV stage size target, KB, 1..64 (default 12) */
    int32_t gemv_stage_kb_interface;
    int32_t coarse_rowblock_min_nrhs; /* row-blocked coarse sweeps from this many columns on, 2..65
                                         (65 = never; default 16) */
    int32_t gemv_rows_interior;       /* streamed-GEMV work unit: row tile of 64, 128 (default) or 256 rows */
    int32_t gemv_rows_interface;
    int32_t coarse_overlap;           /* 1: the interface operator runs on a second stream, concurrently
                                         with the coarse residual and solve (default 0) */
    int32_t sym_stages_interior;      /* shared-memory stages of the symmetric (lower-triangle) GEMV,
                                         3 or 4 (default 4) */
    int32_t sym_stages_interface;
    int32_t interior_block_height;    /* BDDC_LOCAL_SPARSE, one column: the levels of the interior
                                         elimination forest below this height run as per-level gather
                                         sweeps (one warp group per factor row), the levels from it on
                                         supernode by supernode with the node matrices streamed;
                                         0..64, clamped to the forest's levels (default: all levels
                                         in the gather form) */
    int32_t coarse_level_launches;    /* sparse coarse solve, one column: 1 = one launch per level of
                                         the gather form (sub-warp groups per factor row), 0 = one
                                         cooperative launch with grid barriers (default) */
} bddc_tuning_t;

/* Time the candidate launch parameters for blocks of nrhs columns (row
 * tiles of 64, 128 and 256 rows and stage sizes of 6, 12, 24 and 48 KB of
 * the streamed GEMV of each operator family when the handle uses it, or for
 * the symmetric GEMV 3 or 4 stages of 10 to 24 KB;
 * one-row against four-row coarse sweep units when nrhs >= 2; one launch
 * against one launch per level of the one-column coarse sweeps; every split
 * height of the sparse local solver's interior sweeps at one column; whole
 * applies with and without the coarse overlap), apply the fastest and return
 * them in *out (may be NULL).
 * Uses the handle's work vectors (their contents are overwritten) and CUDA
 * events; synchronises `stream`. Results do not change beyond rounding (the
 * candidates differ in scheduling and in the order of some sums). */
int bddc_autotune(bddc_handle_t h, int32_t nrhs, bddc_tuning_t *out, void *stream);
int bddc_get_tuning(bddc_handle_t h, bddc_tuning_t *out);
/* Returns INVALID_ARG (and changes nothing) if a field is out of range. */
int bddc_set_tuning(bddc_handle_t h, const bddc_tuning_t *in);

/* Element term of the adjoint gradient of J(sigma) = 1/2 sum_k ||u_k -
 * u_obs,k||^2 subject to A(sigma) u_k = b_k (the workloads' adjoint
 * configuration; the paper has no gradient): with lambda_k = A^-1 (u_k -
 * u_obs,k) from a second PCG solve on the same handle (A is symmetric),
 *     g[e] = dJ/dsigma_e = - sum_k lambda_k,e^T K_ref u_k,e,
 * K_ref the Q1 stiffness matrix of one element for sigma = 1 and u_k,e,
 * lambda_k,e the 2^dim nodal values of element e. u, lambda: device vectors
 * of n_nodes x nrhs (RHS fastest; Dirichlet entries are treated as 0);
 * g: device array of ne^dim float64, overwritten (element e = ex + ne (ey +
 * ne ez)). Asynchronous on `stream`. */
int bddc_elem_grad(bddc_handle_t h, const double *u, const double *lambda, double *g, int32_t nrhs,
                   void *stream);

/* Solve A x = b by the BDDC-preconditioned conjugate gradient method of
 * Sec. 3 (preconditioner M^-1 of Sec. 2, applied as in bddc_apply) from the
 * start x0 = P_I b (the interior correction of Eq. inner applied to b),
 * independently per column, until ||r_k||_2 <= rtol *
 * ||b||_2 on the updated residual. b, x: device vectors. iters[nrhs] and
 * relres[nrhs] are HOST arrays (may be NULL) receiving the iteration count
 * and ||r||/||b|| of each column. Synchronises `stream`. Returns OK,
 * NOT_CONVERGED or BREAKDOWN. */
int bddc_pcg_solve(bddc_handle_t h, const double *b, double *x, int32_t nrhs,
                   double rtol, int32_t maxit, int32_t *iters, double *relres,
                   void *stream);

/* Same as bddc_pcg_solve with b and x in HOST memory: copies b in, solves
 * and copies x out inside the call (staging through device buffers the
 * handle owns). */
int bddc_pcg_solve_host(bddc_handle_t h, const double *b_host, double *x_host,
                        int32_t nrhs, double rtol, int32_t maxit, int32_t *iters,
                        double *relres, void *stream);

/* Scalars of every iteration of the most recent bddc_pcg_solve(_host) on
 * this handle (Sec. 3: the BDDC-preconditioned CG iteration; per column k:
 * alpha_k = rho_k / p_k^T A p_k, x_k+1 = x_k + alpha_k p_k, r_k+1 = r_k -
 * alpha_k A p_k, beta_k = r_k+1^T z_k+1 / rho_k, or r_k+1^T (z_k+1 - z_k) /
 * rho_k in the flexible forms). rnorm, alpha, beta: HOST arrays (each may
 * be NULL) of (n_iter + 1) * nrhs doubles, entry (k, column j) at k * nrhs
 * + j: rnorm = ||r_k||_2 (r_0 = b - A x_0) for k = 0 .. iters_j; alpha =
 * alpha_k for k < iters_j; beta = the beta computed after iteration k + 1
 * (the one that forms p_k+1) for k < iters_j - 1; NaN elsewhere and for
 * iterations beyond bddc_options_t.history. n_iter must be in [0,
 * history] and nrhs in [1, nrhs_max]. Synchronises the device. */
int bddc_pcg_history(bddc_handle_t h, int32_t nrhs, int32_t n_iter, double *rnorm, double *alpha,
                     double *beta);

/* Copy the coarse residual r_c and the coarse solution u_c = A_c^-1 r_c of
 * the most recent bddc_apply (n_c * nrhs doubles each, coarse dof major,
 * coarse dofs ordered by their smallest node id) into device arrays rc / uc
 * (either may be NULL). Asynchronous on `stream`. */
int bddc_coarse_vectors(bddc_handle_t h, double *rc, double *uc, int32_t nrhs, void *stream);

/* Sizes, byte counts and timings of a handle. */
int bddc_query(bddc_handle_t h, bddc_info_t *info);

/* Device time (milliseconds, CUDA events, median over `reps` applies of the
 * device vector r on `stream`) of each launch of one apply: out_ms[0..8] =
 * restriction, interior operator (t_I = A_II^-1 r_I), condensed interface
 * right-hand side, interface operator (z_G = K_GG y'_G), coarse residual,
 * coarse solve, prolongation, interior right-hand side, interior operator
 * (final). The launches run in sequence, without the coarse overlap of
 * bddc_tuning_t whatever the handle's tuning. For profiling only; z
 * receives M^-1 r. */
int bddc_profile_apply(bddc_handle_t h, const double *r, double *z, int32_t nrhs,
                       int32_t reps, double *out_ms, void *stream);

/* Host-only run of the setup, for inspection and tests: needs no device.
 * With numerics = 0 only the topology runs (subdomain node sets, kappa,
 * globs); otherwise also the float64 local factorisations and the coarse
 * assembly. Fills the size fields of *info (may be NULL) and, if numerics
 * and Ac is not NULL, writes the assembled coarse matrix A_c = sum_i
 * R_ci^T A_ci R_ci (n_c x n_c, row-major, coarse dofs ordered by their
 * smallest node id) when n_c * n_c <= Ac_capacity, else returns
 * INVALID_ARG. Same argument checks and errors as bddc_setup. */
int bddc_setup_inspect(const bddc_problem_t *problem, const bddc_options_t *options,
                       int32_t numerics, bddc_info_t *info, double *Ac, int64_t Ac_capacity);

/* Test hook for the bounded device waits (no counterpart in the paper).
 * With enable = 1, every grid barrier of the sparse coarse solve waits for
 * one arrival more than its grid makes, so the first barrier of every later
 * coarse solve runs out after limit_cycles SM clock cycles (1 .. 4e9; about
 * 2 cycles per ns): the block records BDDC_ERR_TIMEOUT in the handle's
 * device flag and every block of that launch returns (no bulk copy or MMA is
 * in flight in that kernel). The flag then stops PCG (bddc_pcg_solve returns
 * BDDC_ERR_TIMEOUT) and shows in bddc_query().device_error until
 * bddc_clear_device_error. enable = 0 restores the normal barrier and its
 * 2 s limit. Needs the sparse coarse solve (INVALID_ARG otherwise). The
 * handle's captured solve graphs are dropped and captured again. */
int bddc_test_coarse_stall(bddc_handle_t h, int32_t enable, int64_t limit_cycles);

/* Synchronise the handle's device and clear the device error flag that a
 * bounded wait set (bddc_query().device_error). */
int bddc_clear_device_error(bddc_handle_t h);

/* Free the handle and all device memory it holds. NULL is allowed. */
void bddc_destroy(bddc_handle_t h);

/* Static message for a status code. */
const char *bddc_strerror(int status);

/* Detail of the most recent failure on the calling thread ("" if none). */
const char *bddc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BDDC_H */
