// Internal state of a libbddc handle (host side and device side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bddc.h"

namespace bddc {

struct CNodeDev {
  int64_t foff;     // offset of the node's forward matrix [L_PP^-1 ; M]
  int64_t boff;     // offset of the node's backward matrix [L_PP^-T , -M^T]
  int32_t p, u;     // pivots, update-set size
  int32_t pos0;     // elimination position of the first pivot (pivots are contiguous)
  int32_t upd_off;  // offset of the node's update-set dofs
  int32_t fld, bld; // leading dimensions of the two matrices
};
// One warp's unit of a coarse-sweep level: kind 0 = row `row` of L_PP^-1 of
// node `a` (forward), kind 1 = all contributions to the dof at elimination
// position `a` from this level (contributions [b, e)), kind 2 = row `row` of
// the backward matrix of node `a`. In the row-blocked lists (several
// right-hand sides) kinds 0 and 2 cover rows [row, row + b).
struct CUnit {
  int32_t kind, a, row, b, e;
};
// One output value of a coarse sweep in the gather form (one right-hand
// side): value = sum_{j < len} C[off + j] * X[I[off + j]], where an index
// below n_c addresses the first operand vector and an index n_c + i entry i
// of the second (forward: r' in elimination order, r_c in dof order;
// backward: y, u in elimination order). Forward: aux < 0 writes y[dst]; aux
// >= 0 writes r'[dst] = X[aux] - value. Backward: writes u at position dst
// and at dof aux.
struct CGUnit {
  int64_t off;
  int32_t len, dst, aux, pad;
};
// The gather form of both sweeps (built on the host in coarse_sparse.cpp,
// applied by coarse_solve.cu): C and I hold each
// unit's coefficients and operand indices contiguously; for each launch shape
// s (blocks[s] x warps_per_block[s] warps, warp w of block b being warp
// b * warps_per_block[s] + w) the descriptors of warp w in phase ph are
// units[s][wo[s][ph (warps+1) + w] .. wo[s][ph (warps+1) + w + 1]), processed
// in that order. Phases 0 .. L-1 are the forward levels (height = phase),
// phases L .. 2L-1 the backward levels (height = 2L-1-phase); with a dense
// top of k levels, phases 0 .. L-k-1 are the forward levels below it, phase
// L-k the dense product, then the backward levels from height L-k-1 down.
struct CoarseFactor;
constexpr int kLocalLeaf = 32;      // default leaf size of the interior factorisations
constexpr int kGatherBatch = 256;   // coefficients a warp reads per step of a unit (cost unit of the assignment)
constexpr long long kBarrierWaitCycles = 4000000000LL;   // grid-barrier wait limit: about 2 s at 2 GHz
struct GatherLayout {
  std::vector<double> C;
  std::vector<int32_t> I;
  std::vector<std::vector<CGUnit>> units;
  std::vector<std::vector<int32_t>> wo;
  // every phase's descriptors in storage order (longest unit first), phase
  // ph at [seq_off[ph], seq_off[ph + 1]): the per-level launches
  std::vector<CGUnit> seq;
  std::vector<int64_t> seq_off;
  // phases: fwd_phases forward-type phases (the forward levels, then the
  // dense top's product if the factor has one), then the backward levels
  int fwd_phases = 0, phases = 0;
};
void gather_layout(const CoarseFactor& cf, int nshapes, const int* blocks, const int* warps_per_block,
                   GatherLayout& g);
// One contribution to a receiving dof: an M row of a node and its operand.
struct CContrib {
  int64_t row_off;  // offset of the M row in the forward matrices
  int32_t x_off;    // elimination position of the node's first pivot
  int32_t len;      // p of the node
  int64_t pad;
};
// Block form of the one-column sweeps: one supernode and one chunk of its
// rows (see BlockLayout below).
struct SNode {
  int64_t foff, boff;     // F: (p + u) x fld, B: p x bld (row-major)
  int32_t p, u, pos0;
  int32_t fld, bld;
  int32_t cbase;          // this node's contribution vector c (u values) in the contribution buffer
  int32_t cmap0;          // its map into the parent's front (u indices)
  int32_t kid0, nkid;     // children: kids[kid0 .. kid0 + nkid)
  int32_t upd_off;        // positions of the update set: upd[upd_off .. upd_off + u)
  int32_t height;         // height in the elimination tree (leaves 0)
};
struct BlockItem {
  int32_t node, row0, nrows, g;
};
// Device form of one supernodal factorisation and of its sweeps
// (coarse_solve.cu): the coarse factor of A_c, or the forest of the
// interior factors of all subdomains (sparse local solver). F, B: node
// matrices (several right-hand sides); gC, gI, gU, gwo: the gather form (one
// right-hand side) for launch shapes [0] blocks of 512 threads and [1] of
// 256; bar: the persistent kernel's grid-barrier counter.
struct SweepSet {
  double* F = nullptr;          // forward matrices [L_PP^-1 ; M]
  double* B = nullptr;          // backward matrices [L_PP^-T , -M^T]
  CNodeDev* nodes = nullptr;
  CUnit* units = nullptr;       // warp units, forward levels then backward levels
  CUnit* units4 = nullptr;      // the same with kinds 0 and 2 blocked by 4 rows
  CContrib* list = nullptr;     // contributions of the receiving units
  int32_t* upd = nullptr;       // update-set dofs of every node
  int32_t* order = nullptr;     // elimination position -> dof
  int32_t* lvl = nullptr;       // unit offsets: [L+1 forward][L+1 backward], then n
  int32_t* lvl4 = nullptr;
  double* gC = nullptr;
  float* gC32 = nullptr;        // the gather form's coefficients in float32 (per-level form only), else null
  float* x32 = nullptr;         // with gC32: float32 copies of r', y and r (n each), the operands the sweeps read
  int32_t* gI = nullptr;
  CGUnit* gU[2] = {nullptr, nullptr};
  int32_t* gwo[2] = {nullptr, nullptr};   // [phases][warps + 1]
  unsigned int* bar = nullptr;
  int64_t n = 0;                // dofs
  int levels = 0, grid = 0, grid4 = 0, g_blocks = 0;
  int g_fwd = 0, g_phases = 0;  // gather form: forward-type phases, all phases
  int64_t nnz = 0;              // stored entries of F and B
  int64_t g_entries = 0;        // stored entries of the gather form
  int64_t update_total = 0;     // sum of the update-set sizes
  bool multi = false;           // F, B and the unit lists built (several right-hand sides)
  // per-level form (one right-hand side, large factors): one launch per
  // phase; a phase's units are in classes of decreasing length, class c
  // processed by groups of kLevelGroup[c] lanes: units [cb[c], cb[c+1]) of
  // the phase's descriptors (seq + u0), blocks [bb[c], bb[c+1]) of its grid
  struct LevelPhase {
    int64_t u0;
    int32_t cb[7], bb[7];
  };
  CGUnit* seq = nullptr;
  std::vector<LevelPhase> lv;
  bool use_level = false;       // one column: the per-level form (else the cooperative launch)
  // block form (one right-hand side, large factors; see BlockLayout): node
  // records, children, maps into the parents' fronts, update positions,
  // work items per phase, the contribution buffer; F and B above
  bool block_form = false;
  SNode* bnodes = nullptr;
  int32_t* bkids = nullptr;
  int32_t* bcmap = nullptr;
  int32_t* bupd = nullptr;
  BlockItem* bitems = nullptr;
  double* cbuf = nullptr;
  std::vector<int64_t> bitem_off;
  int block_min_height = 0;        // levels below this height run the per-level gather form
  std::vector<int64_t> bn_big;     // per phase: items that are chunks of large nodes (listed first)
  std::vector<int> bphase_front;   // largest front of each phase's large nodes
  int64_t read_1col = 0;           // bytes of coefficients and indices one one-column solve of the gather form reads
  std::vector<int64_t> gbytes_h, bbytes_h;   // the same per height: gather form, block form
};
// Bytes of coefficients (and indices) one one-column solve reads in the
// form the set runs (the block form's split included).
inline int64_t sweep_read_1col(const SweepSet& S) {
  if (!S.block_form) return S.read_1col;
  const int k = S.block_min_height < 0 ? 0 : S.block_min_height > S.levels ? S.levels : S.block_min_height;
  int64_t b = 0;
  for (int lv = 0; lv < S.levels; ++lv) b += lv < k ? S.gbytes_h[lv] : S.bbytes_h[lv];
  return b;
}
// forms of the one-column sweeps (build_sweeps)
constexpr int kSweepCoop = 0;       // gather form, one cooperative launch (small factors)
constexpr int kSweepLevel = 1;      // gather form, one launch per phase
constexpr int kSweepBlock = 2;      // block form, one launch per phase (large factors)
constexpr int64_t kBlockTarget = 8192;   // matrix entries per work item of the block form
constexpr int kSmallFront = 128;         // fronts up to this size: one warp per node (8 per block)
constexpr int kBlockMaxFront = 16384;    // largest front of the block form (shared memory)
constexpr int kLevelThreads = 256;
constexpr int kLevelClasses = 6;
constexpr int kLevelGroup[kLevelClasses] = {32, 16, 8, 4, 2, 1};
// The class of a unit of len coefficients: groups of 32, 16, 8, 4, 2 and 1
// lanes from 512, 192, 80, 32 and 12 coefficients on, i.e. 12 to 16 of them
// per lane at most (measured on the interior sweeps of the 2D workloads, in
// float64 and float32: groups twice as wide took 1.2 to 1.5x as long, half
// as wide 1.04 to 1.11x; more units per warp hide the load latency, and
// every shuffle step of a group's sum costs the float64 pipe)
inline int level_class(int len) {
  if (len >= 512) return 0;
  if (len >= 192) return 1;
  if (len >= 80) return 2;
  if (len >= 32) return 3;
  if (len >= 12) return 4;
  return 5;
}
// The per-level form of a gather layout (seq, seq_off): every phase's class
// ranges and block counts (kLevelThreads / G units per block of class G).
void level_phases(const GatherLayout& g, std::vector<SweepSet::LevelPhase>& out);

// Block form of the one-column sweeps (large factors; dofs numbered in
// elimination order): supernode by supernode, with the node's dense
// matrices streamed row by row. Forward, node t: its front f (p + u values)
// = r at its pivots plus its children's contribution vectors (each child's
// update set mapped into t's front, children in order); y_P = L_PP^-1 f_P
// and the contribution c_t = f_U - M f_P (rows of F). Backward: u_P = [L_PP^-T,
// -M^T] [y_P; u_U] (rows of B), u_U read at the update set's positions.
// A work item is a chunk of rows of one node, processed by one block with
// `g` lanes per row.
struct BlockLayout {
  std::vector<SNode> nodes;
  std::vector<int32_t> kids, cmap, upd;
  std::vector<BlockItem> items;       // forward levels (height 0 first), then backward levels
  std::vector<int64_t> item_off;      // 2 L + 1 phase offsets into items
  std::vector<int64_t> n_big;         // per phase: its first n_big items are chunks of large nodes
                                      // (one block each); the rest are whole small nodes (one warp each)
  std::vector<double> F, B;
  int64_t cbuf = 0;                   // contribution buffer size (sum of u)
  int max_front = 0;                  // largest p + u
};
// Builds the block form of cf (which must be renumbered: order = identity):
// nodes whose front has more than kSmallFront values in chunks of about
// target_entries matrix entries, the others whole.
void block_layout(const CoarseFactor& cf, int64_t target_entries, BlockLayout& out);
inline int block_group(int len) { return len >= 128 ? 32 : len >= 48 ? 16 : len >= 20 ? 8 : 4; }

// Tensor-core batched GEMM (bddc_tc_gemm.cu). A dense n x n operator is
// stored as chunks of up to 128 rows x kTcChunkK(precision) columns in the
// canonical no-swizzle K-major layout of tcgen05.mma: core matrices of 8 rows
// x 16 bytes, ordered [8-row group][16-byte column slice][8 rows][16 bytes],
// so the valid rows of a chunk are one contiguous prefix. One unit is up to
// kTcGroup row tiles of one operator; its chunks are stored in stream order
// (column chunk outer, row tile inner).
constexpr int kTcRows = 128;      // rows per tile (MMA M)
constexpr int kTcGroup = 8;       // row tiles per unit (TMEM: 8 x N <= 512 columns)
constexpr int kTcMinRhs = 8;      // nrhs_max from which the BF16 form uses tensor cores
struct TcUnit {
  int64_t aoff;   // element offset of the unit's first chunk in the tiled arena
  int32_t n;      // operator dimension
  int32_t g;      // row tiles in the unit
  int32_t row0;   // first row of the unit
  int32_t xoff;   // first entry of the operand in the compact X buffer
  int32_t yoff;   // first entry of the result in the compact Y buffer
  int32_t kbase;  // first column of the operator in the packed operand buffer
};

// One row tile of one dense operator in a batched GEMV launch:
// Y[yoff + row0 + r] = sum_c Op[row0 + r, c] * X[xoff + c], r < nrows.
struct WorkItem {
  int64_t moff;    // element offset of the operator (row 0) in its arena
  int32_t lda;     // leading dimension (elements), padded to 16 bytes
  int32_t ncols;   // operator columns (= rows of the square operator)
  int32_t row0;    // first row of this tile
  int32_t nrows;   // rows in this tile
  int32_t xoff;    // first entry of the operand in the compact X buffer
  int32_t yoff;    // first entry of the result in the compact Y buffer
};

// One supernode of the sparse Cholesky factorisation of A_c (coarse_sparse.cpp).
struct CoarseNode {
  std::vector<int32_t> piv;     // pivot coarse dofs (the separator, or a leaf's set)
  std::vector<int32_t> upd;     // update set: later coarse dofs coupled to the subtree
  std::vector<int> children;
  int parent = -1, first = 0, last = -1, height = 0, p = 0, u = 0;
  std::vector<double> Fm;       // (p+u) x p: [L_PP^-1 ; M],   M = L_UP L_PP^-1
  std::vector<double> Bm;       // p x (p+u): [L_PP^-T , -M^T]
};
struct CoarseFactor {
  int64_t n = 0;
  std::vector<CoarseNode> nodes; // post-order
  std::vector<int32_t> order;    // elimination position -> coarse dof
  int n_levels = 0;              // 1 + largest node height (leaves have height 0)
  int64_t nnz = 0;               // stored entries of one sweep's matrices
  // dense top (optional): the dofs of the nodes of the top `top_levels`
  // levels (T, closed under ancestors; elimination positions, ascending) and
  // the inverse of their Schur complement S_TT = A_TT - A_TB A_BB^-1 A_BT,
  // which equals (A^-1)_TT: one dense product replaces the sweeps of those
  // levels
  int top_levels = 0;
  std::vector<int32_t> top_pos;
  std::vector<double> top_inv;   // |T| x |T|, row-major
};
constexpr int64_t kCoarseDenseTop = 2048;   // largest dense top of the coarse factor
// Nested-dissection supernodal Cholesky of the SPD matrix (rp, ci, val)
// (CSR, both triangles); xyz: 3 coordinates per dof for the dissection.
// dof_subs: the subdomains of every coarse dof (glob); sub_xyz: centroid of
// every subdomain (3 per subdomain) for the dissection.
// Renumbers the coarse dofs of a factorisation by their elimination
// position (pivot and update-set lists; the order becomes the identity);
// perm[old dof] = new dof.
void coarse_renumber(CoarseFactor& cf, std::vector<int32_t>& perm);
// top_max > 0: the most top levels (at least one level left below) whose
// dofs number at most top_max become a dense top (see CoarseFactor).
int coarse_factor(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& val, const std::vector<std::vector<int32_t>>& dof_subs,
                  const std::vector<double>& sub_xyz, CoarseFactor& cf, std::string& err, int64_t top_max = 0);
// The same factorisation in general form (coarse_factor is the case n_keep
// = 0, leaf 384): the dofs [0, n - n_keep) are ordered by nested dissection
// of their groups (dof_groups: the groups holding each of them; group_xyz: 3
// coordinates per group) with vertex sets up to `leaf` dofs not split, and
// factorised; the kept dofs [n - n_keep, n) are eliminated last as one front
// that is assembled but not factorised: it is their Schur complement,
// returned in *schur (n_keep x n_keep, row-major). The factor holds the
// eliminated dofs alone (n = n - n_keep; the kept dofs are dropped from the
// update sets).
int sparse_factor(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& val, const std::vector<std::vector<int32_t>>& dof_groups,
                  const std::vector<double>& group_xyz, int64_t n_keep, int leaf, CoarseFactor& cf,
                  std::vector<double>* schur, std::string& err, int64_t top_max = 0);
// One factorisation of the block-diagonal matrix diag(parts): part s holds
// dofs and positions [off[s], off[s] + parts[s].n) (a forest of elimination
// trees whose levels are merged by height).
void merge_forest(const std::vector<CoarseFactor>& parts, const std::vector<int32_t>& off, CoarseFactor& out);

// Host-side results of the topology and numeric setup (float64).
struct HostSetup {
  int dim = 0, ne = 0, n1 = 0;
  int64_t n_nodes = 0, n_elems = 0;
  double h = 0;
  int n_sub = 0;
  // Dirichlet nodes and multiplicity kappa per node (0 on Dirichlet nodes)
  std::vector<int32_t> dir_nodes;
  std::vector<uint8_t> kappa;
  // per subdomain: interior and interface nodes (sorted node ids)
  std::vector<std::vector<int32_t>> sub_I, sub_G;
  // globs: members (node ids), sharing subdomains, kind (CORNER/EDGE/FACE)
  std::vector<std::vector<int32_t>> glob_nodes, glob_subs;
  std::vector<int> glob_kind;
  std::vector<std::vector<int32_t>> sub_globs;   // glob ids per subdomain, ascending
  // per subdomain numeric results
  std::vector<std::vector<double>> AIIinv;   // nI x nI
  std::vector<std::vector<double>> Kgg;      // nG x nG: (1,1) block of the constrained Schur KKT inverse
  std::vector<std::vector<double>> Phi;      // nG x nc: interface rows of Phi_i
  std::vector<std::vector<double>> Aci;      // nc x nc
  // sparse couplings, CSR: A_GI (rows: local interface, cols: local interior)
  std::vector<std::vector<int32_t>> agi_ptr, agi_col, aig_ptr, aig_col;
  std::vector<std::vector<double>> agi_val, aig_val;
  // coarse operator
  int64_t n_c = 0;
  bool coarse_dense = true;                  // dense inverse (else the sparse factor or CG)
  bool coarse_cg = false;                    // inexact coarse solve by plain CG on A_c
  std::vector<double> Acinv;                 // n_c x n_c dense inverse (dense mode)
  std::vector<int64_t> Ac_ptr;               // A_c in CSR (both triangles)
  std::vector<int32_t> Ac_col;
  std::vector<double> Ac_val;
  CoarseFactor cfac;                         // its sparse Cholesky factorisation
  // sparse local solver: per subdomain, the factorisation of A_II (dofs in
  // local interior order)
  bool sparse_local = false;
  std::vector<CoarseFactor> ifac;
  int error_subdomain = -1;
};

// The work vectors of one apply (each nrhs columns wide, right-hand side
// fastest): compact interior (rI, tI, bI), interface copies (yG, zG, eG),
// local constraints (g), coarse (rc, uc), and the coarse solve's own: r' and y
// of the factor's sweeps or r and p of the coarse CG (cr, cy), A_c p of the
// coarse CG (cq), the dense coarse solve's panel products (cpart), and r'
// and y of the interior factors' sweeps (ir, iy).
struct ApplyWork {
  double *rI = nullptr, *tI = nullptr, *bI = nullptr;
  double *yG = nullptr, *zG = nullptr, *eG = nullptr;
  double *g = nullptr, *rc = nullptr, *uc = nullptr;
  double *cr = nullptr, *cy = nullptr, *cq = nullptr, *cpart = nullptr;
  double *ir = nullptr, *iy = nullptr;   // r' and y of the interior sweeps (sparse local solver)
};

// Makes `device` current for the lifetime of the guard and restores the
// caller's current device afterwards (every entry point of the C ABI).
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      return;
    }
    ok = prev == device || cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Record `msg` for bddc_last_error() on this thread; returns `code`.
int set_last_error(int code, const std::string& msg);

// Validate the problem and options (no device checks).
int validate_problem(const bddc_problem_t* p, const bddc_options_t* o, std::string& err);
// Topology and float64 numerics; with factor_coarse = false A_c is assembled
// but not factorised.
int host_setup(const bddc_problem_t* p, const bddc_options_t* o, HostSetup& hs, std::string& err,
               bool factor_coarse = true, bool numerics = true);

}  // namespace bddc

struct bddc_handle_s {
  // problem
  int dim = 0, ne = 0, n1 = 0, n_sub = 0, precision = 0, nrhs_max = 1, device = 0;
  bool use_graph = true;
  // launch parameters chosen by the autotuner (or set by the caller)
  int tune_stage_kb[2] = {12, 12};   // streamed GEMV stage size: interior, interface operators
  int tune_sym_stages[2] = {4, 4};   // stages of the symmetric GEMV: interior, interface operators
  int tune_tile_class[2] = {1, 1};   // streamed GEMV row tile 64 << class: interior, interface
  int tune_coarse_rb_min = 16;       // row-blocked coarse sweeps from this many right-hand sides on
  int tune_overlap = 0;              // interface operator concurrent with the coarse residual and solve
  // second stream of the apply and its fork / join events, one set per
  // capture sequence: [0] direct launches and the solve graph's prologue,
  // [1] the body of its conditional node (captured while [0] is still open)
  cudaStream_t aux_stream[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};
  int aux_sel = 0;
  int64_t n_nodes = 0, n_elems = 0;
  double h = 0;
  // sizes
  int64_t nI_tot = 0, nG_tot = 0, nC_tot = 0, n_c = 0, n_gu = 0, n_dir = 0;
  bddc_info_t info{};
  // --- device data ---------------------------------------------------
  double* d_sigma = nullptr;          // [n_elems]
  int32_t* d_dnode = nullptr;         // [n_dir] Dirichlet nodes
  int32_t* d_inode = nullptr;         // [nI_tot] node of each compact interior entry
  int32_t* d_gnode = nullptr;         // [nG_tot] node of each interface copy
  double* d_gw = nullptr;             // [nG_tot] 1/kappa of each interface copy
  // A_GI: rows = interface copies, cols = compact interior positions
  int32_t* d_agi_ptr = nullptr; int32_t* d_agi_col = nullptr; double* d_agi_val = nullptr;
  // A_IG: rows = compact interior positions, cols = node ids (interface nodes)
  int32_t* d_aig_ptr = nullptr; int32_t* d_aig_col = nullptr; double* d_aig_val = nullptr;
  // Phi_Gamma^T [nc x nG] per subdomain (phi_prec), with the work list of the
  // coarse residual's streamed GEMV; the prolongation reads it column-wise
  void* d_phit = nullptr;             // Phi_G^T arena (phi_prec)
  int phi_prec = BDDC_PREC_FP64;      // BDDC_PREC_FP64 or BDDC_PREC_FP32
  bddc::WorkItem* d_wi_PT = nullptr; int n_wi_PT = 0; int max_ld_PT = 0;
  int64_t* d_pt_off = nullptr;        // [n_sub] element offset of each subdomain's Phi_G^T block
  int32_t* d_pt_ld = nullptr;         // [n_sub] its leading dimension
  int32_t* d_sub_goff = nullptr;      // [n_sub + 1] interface copy offsets
  int32_t* d_sub_coff = nullptr;      // [n_sub + 1] local constraint offsets
  int32_t* d_csub = nullptr;          // [nC_tot] subdomain of each local constraint
  int32_t* d_ccdof = nullptr;         // [nC_tot] coarse dof of each local constraint
  // coarse gather: per coarse dof, the local-constraint positions that sum into it
  int32_t* d_cg_ptr = nullptr; int32_t* d_cg_idx = nullptr;
  // prolongation: per unique interface node, its copies
  int32_t* d_gu_node = nullptr; int32_t* d_gu_ptr = nullptr; int32_t* d_gu_copy = nullptr;
  // operators
  void* d_aii = nullptr;              // interior inverses, precision-typed arena
  void* d_kgg = nullptr;              // interface operators, precision-typed arena
  // dense coarse solve: A_c^-1 in column panels, streamed GEMV + panel sum
  bool coarse_dense = true;
  double* d_acinv = nullptr;
  int32_t ldc = 0, n_cpanels = 0;
  bddc::WorkItem* d_wi_C = nullptr; int n_wi_C = 0;
  // sparse coarse solve (coarse_solve.cu): the coarse factor's sweeps
  bddc::SweepSet cs;
  int32_t* d_cperm = nullptr;         // glob -> device coarse dof (sparse coarse: elimination order)
  unsigned int* d_cbar = nullptr;     // grid barrier of the persistent coarse kernels
  int g_blocks = 0;                   // requested grid of the one-column coarse sweeps (0 = SMs)
  int c_sms = 0;
  int64_t c_nnz = 0;                  // stored entries of the coarse operator
  // sparse local solver: the interior factors of all subdomains as one forest
  // (dofs = compact interior positions, numbered in elimination order)
  bool sparse_local = false;
  bddc::SweepSet is;
  // inexact coarse solve by CG: A_c in CSR (glob order), work vectors, block partials
  bool coarse_cg = false;
  int32_t* d_acp = nullptr; int32_t* d_acc = nullptr; double* d_acv = nullptr;
  double* d_cgpart = nullptr;          // [c_sms][2][nrhs_max]
  int32_t* d_cgiters = nullptr;        // [nrhs_max] iterations of the last coarse solve
  int cg_maxit = 2000;
  double cg_rtol = 1e-10;
  bddc::WorkItem* d_wi_I = nullptr; int n_wi_I = 0;
  bddc::WorkItem* d_wi_G = nullptr; int n_wi_G = 0;
  // larger row tiles for the streamed (bulk-copy) GEMV
  // streamed-GEMV work lists for row tiles of 64 << c rows, c = 0, 1, 2
  bddc::WorkItem* d_wtx_I[3] = {nullptr, nullptr, nullptr}; int n_wtx_I[3] = {0, 0, 0};
  bddc::WorkItem* d_wtx_G[3] = {nullptr, nullptr, nullptr}; int n_wtx_G[3] = {0, 0, 0};
  bool use_tma = false;
  // symmetric operators as packed lower triangles (one work item per operator)
  bool use_sym = false;
  bool full_operators = false;        // option: keep them in full
  bddc::WorkItem* d_wsy_I = nullptr; int n_wsy_I = 0;
  bddc::WorkItem* d_wsy_G = nullptr; int n_wsy_G = 0;
  int max_n_I = 0, max_n_G = 0;
  // tensor-core path: tiled arenas (d_aii / d_kgg then hold the tiled layout)
  bool use_tc = false;
  bddc::TcUnit* d_tcu_I = nullptr; int n_tcu_I = 0;
  bddc::TcUnit* d_tcu_G = nullptr; int n_tcu_G = 0;
  int32_t* d_tcs_I = nullptr; int64_t n_tcs_I = 0;   // operand slice -> operator (interior)
  int32_t* d_tcs_G = nullptr; int64_t n_tcs_G = 0;
  int32_t* d_tcop_I = nullptr; int32_t* d_tcop_G = nullptr;   // per operator: {xoff, n, kbase, slice0}
  void* d_tcB = nullptr;               // packed operand (hi/lo), sized for the widest nrhs
  int64_t tcB_cols_I = 0, tcB_cols_G = 0;   // sum of padded operator widths
  int tc_maxg_I = 0, tc_maxg_G = 0;          // most row tiles in one unit
  int max_cols_I = 0, max_cols_G = 0;
  int max_nc = 0;                     // most constraints of one subdomain
  // apply workspace (nrhs_max columns)
  bddc::ApplyWork w;                  // the apply's work vectors (nrhs_max columns)
  // PCG workspace
  double *p_r = nullptr, *p_z = nullptr, *p_zold = nullptr, *p_p = nullptr, *p_q = nullptr;
  double *s_b = nullptr, *s_x = nullptr;   // staging for host-buffer solves
  double* d_partials = nullptr;            // [n_red_blocks * nrhs_max * 3]
  double* d_scal = nullptr;                // per-column PCG scalars
  int32_t* d_iscal = nullptr;              // per-column flags / counters
  int32_t* h_flags = nullptr;              // pinned host mirror of the global flags
  int32_t* d_err = nullptr;                // device error flag (inside d_iscal)
  double* d_hist = nullptr;                // [3][hist_cap + 1][nrhs_max] PCG history (null if not kept)
  int hist_cap = 0;                        // iterations whose scalars are kept
  // fault injection for tests of the bounded waits: the coarse solve's grid
  // barriers wait for cbar_extra arrivals more than the grid makes, with a
  // wait limit of cbar_cycles clock cycles
  unsigned int cbar_extra = 0;
  long long cbar_cycles = bddc::kBarrierWaitCycles;
  int n_red_blocks = 0;
  double* d_stencil = nullptr;             // [stencil points][n_nodes] assembled Q1 stencil
  unsigned int* d_counter = nullptr;       // blocks finished in the current reducing kernel
  // one PCG iteration captured as a CUDA graph, valid for (x, nrhs, rtol, form)
  cudaGraphExec_t iter_graph = nullptr;
  const double* graph_x = nullptr;
  int graph_nrhs = 0, graph_flexible = -1;
  double graph_rtol = 0.0;
  int64_t graph_launches = 0;              // kernels in one replay
  // the whole solve as one graph: prologue and first iteration, then a
  // conditional WHILE node over one iteration; valid for (b, x, nrhs, rtol, maxit, form)
  cudaGraphExec_t solve_graph = nullptr;
  const double* solve_b = nullptr;
  const double* solve_x = nullptr;
  int solve_nrhs = 0, solve_maxit = 0, solve_flexible = -1;
  double solve_rtol = 0.0;
  int64_t solve_pro_launches = 0, solve_body_launches = 0;
  cudaStream_t body_stream = nullptr;
  bool solve_graph_unsupported = false;
  cudaStream_t cap_stream = nullptr;       // private stream used only for capture
  int64_t launches = 0;                    // kernels launched so far
  std::vector<void*> allocations;
};
