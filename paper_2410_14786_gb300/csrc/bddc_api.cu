// C ABI of libbddc: setup upload, apply, matvec, PCG driver.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/bddc.h"
#include "internal.hpp"
#include "kernels.cuh"

using namespace bddc;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? BDDC_ERR_OOM : BDDC_ERR_CUDA,               \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

template <typename T>
cudaError_t dev_alloc(bddc_handle_s* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T));
  if (e == cudaSuccess) {
    h->allocations.push_back(v);
    *p = static_cast<T*>(v);
  }
  return e;
}

template <typename T>
cudaError_t upload(bddc_handle_s* h, T** p, const std::vector<T>& v) {
  cudaError_t e = dev_alloc(h, p, v.size());
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// The local operators run on the tensor cores for BF16 and TF32 when asked,
// or (AUTO) when blocks of at least kTcMinRhs right-hand sides are expected.
bool tc_enabled(const bddc_options_t* O) {
  return (O->precision == BDDC_PREC_TF32 || O->precision == BDDC_PREC_BF16) &&
         (O->tensor_cores == BDDC_TC_ON || (O->tensor_cores == BDDC_TC_AUTO && O->nrhs_max >= kTcMinRhs));
}

// The precision the operators are stored and applied in: a TF32 request
// that AUTO keeps off the tensor cores (fewer than kTcMinRhs right-hand
// sides, where an MMA of N = 16 would waste most of its work) runs the FP32
// form on the CUDA cores.
int effective_precision(const bddc_options_t* O) {
  return O->precision == BDDC_PREC_TF32 && !tc_enabled(O) ? BDDC_PREC_FP32 : O->precision;
}

int elem_bytes(int precision) {
  return precision == BDDC_PREC_FP64 ? 8 : (precision == BDDC_PREC_FP32 || precision == BDDC_PREC_TF32) ? 4 : 2;
}

// leading dimension padded so that every row starts on a 16-byte boundary
int32_t padded_ld(int n, int eb) {
  const int v = 16 / eb;
  return (int32_t)((n + v - 1) / v * v);
}

// Pack per-subdomain dense operators (float64 on the host) into one arena
// of the target precision; block starts aligned to 256 bytes.
template <typename T>
std::vector<T> pack_arena(const std::vector<std::vector<double>>& ops, const std::vector<int>& dims,
                          std::vector<int64_t>& off, std::vector<int32_t>& ld, T (*cvt)(double)) {
  const int eb = (int)sizeof(T);
  const int64_t align = 256 / eb;
  off.assign(ops.size(), 0);
  ld.assign(ops.size(), 0);
  int64_t cur = 0;
  for (size_t s = 0; s < ops.size(); ++s) {
    cur = (cur + align - 1) / align * align;
    off[s] = cur;
    ld[s] = padded_ld(dims[s], eb);
    cur += (int64_t)dims[s] * ld[s];
  }
  std::vector<T> out((size_t)std::max<int64_t>(cur, 1), cvt(0.0));
  for (size_t s = 0; s < ops.size(); ++s) {
    const int n = dims[s];
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) out[off[s] + (int64_t)r * ld[s] + c] = cvt(ops[s][(size_t)r * n + c]);
  }
  return out;
}

// Pack per-subdomain symmetric operators as their lower triangles: row g
// holds columns 0 .. g (entries averaged with their transposes, the diagonal
// halved), zero-padded to 16 bytes; blocks aligned to 256 bytes. The
// operator is L' + L'^T.
template <typename T>
std::vector<T> pack_lower(const std::vector<std::vector<double>>& ops, const std::vector<int>& dims, int prec,
                          std::vector<int64_t>& off, T (*cvt)(double)) {
  const int64_t align = 256 / (int)sizeof(T);
  off.assign(ops.size(), 0);
  int64_t cur = 0;
  for (size_t s = 0; s < ops.size(); ++s) {
    cur = (cur + align - 1) / align * align;
    off[s] = cur;
    cur += sym_packed_elems(prec, dims[s]);
  }
  std::vector<T> out((size_t)std::max<int64_t>(cur, 1), cvt(0.0));
  for (size_t s = 0; s < ops.size(); ++s) {
    const int n = dims[s];
    const std::vector<double>& A = ops[s];
    for (int g = 0; g < n; ++g) {
      T* row = &out[off[s] + sym_packed_elems(prec, g)];
      for (int c = 0; c < g; ++c) row[c] = cvt(0.5 * (A[(size_t)g * n + c] + A[(size_t)c * n + g]));
      row[g] = cvt(0.5 * A[(size_t)g * n + g]);
    }
  }
  return out;
}

// Pack per-subdomain rectangular float64 blocks (rows x cols, row-major on
// the host) with rows padded to 16 bytes of the storage type (eb bytes per
// element) and blocks aligned to 32 elements.
std::vector<double> pack_rect(const std::vector<std::vector<double>>& src, const std::vector<int>& rows,
                              const std::vector<int>& cols, bool transpose, int eb, std::vector<int64_t>& off,
                              std::vector<int32_t>& ld) {
  // transpose: src[s] is cols x rows and the block stores its transpose
  const size_t S = rows.size();
  off.assign(S, 0);
  ld.assign(S, 0);
  int64_t cur = 0;
  for (size_t s = 0; s < S; ++s) {
    cur = (cur + 31) / 32 * 32;
    off[s] = cur;
    ld[s] = padded_ld(cols[s], eb);
    cur += (int64_t)rows[s] * ld[s];
  }
  std::vector<double> out((size_t)std::max<int64_t>(cur, 1), 0.0);
  for (size_t s = 0; s < S; ++s)
    for (int r = 0; r < rows[s]; ++r)
      for (int c = 0; c < cols[s]; ++c)
        out[off[s] + (int64_t)r * ld[s] + c] =
            transpose ? src[s][(size_t)c * rows[s] + r] : src[s][(size_t)r * cols[s] + c];
  return out;
}

// The streamed GEMV moves operator rows with 16-byte bulk copies and reads
// them with 16-byte vector loads: every item must start on, and have a row
// pitch of, a multiple of 16 bytes.
bool items_aligned(const std::vector<WorkItem>& items, int eb) {
  for (const WorkItem& w : items)
    if ((w.moff * eb) % 16 != 0 || ((int64_t)w.lda * eb) % 16 != 0 || w.lda < w.ncols) return false;
  return true;
}

// Row tiles of rectangular operators.
std::vector<WorkItem> make_rect_items(const std::vector<int64_t>& off, const std::vector<int32_t>& ld,
                                      const std::vector<int>& rows, const std::vector<int>& cols,
                                      const std::vector<int32_t>& xoff, const std::vector<int32_t>& yoff, int tile) {
  std::vector<WorkItem> items;
  for (size_t s = 0; s < rows.size(); ++s)
    for (int r0 = 0; r0 < rows[s]; r0 += tile)
      items.push_back(WorkItem{off[s], ld[s], cols[s], r0, std::min(tile, rows[s] - r0), xoff[s], yoff[s]});
  std::stable_sort(items.begin(), items.end(),
                   [](const WorkItem& a, const WorkItem& b) { return a.ncols > b.ncols; });
  return items;
}

double cvt_d(double v) { return v; }
float cvt_f(double v) { return (float)v; }
__nv_bfloat16 cvt_b(double v) { return __float2bfloat16_rn((float)v); }

// Row tiles of square operators: (offset, ld, n, x/y offset) per subdomain.
std::vector<WorkItem> make_items(const std::vector<int64_t>& off, const std::vector<int32_t>& ld,
                                 const std::vector<int>& dims, const std::vector<int32_t>& voff, int tile) {
  std::vector<WorkItem> items;
  for (size_t s = 0; s < dims.size(); ++s)
    for (int r0 = 0; r0 < dims[s]; r0 += tile)
      items.push_back(WorkItem{off[s], ld[s], dims[s], r0, std::min(tile, dims[s] - r0), voff[s], voff[s]});
  // largest operators first: long tiles start early
  std::stable_sort(items.begin(), items.end(),
                   [](const WorkItem& a, const WorkItem& b) { return a.ncols > b.ncols; });
  return items;
}

int build_device(bddc_handle_s* h, HostSetup& hs, const bddc_problem_t* P) {
  const int S = hs.n_sub;
  int64_t in_coarse_bytes = 0, coarse_read_1rhs = 0;
  // ---- compact layouts --------------------------------------------------------
  std::vector<int32_t> ioff(S + 1, 0), goff(S + 1, 0), coff(S + 1, 0);
  for (int s = 0; s < S; ++s) {
    ioff[s + 1] = ioff[s] + (int32_t)hs.sub_I[s].size();
    goff[s + 1] = goff[s] + (int32_t)hs.sub_G[s].size();
    coff[s + 1] = coff[s] + (int32_t)hs.sub_globs[s].size();
    h->max_nc = std::max(h->max_nc, (int)hs.sub_globs[s].size());
  }
  h->nI_tot = ioff[S]; h->nG_tot = goff[S]; h->nC_tot = coff[S]; h->n_c = hs.n_c;
  h->n_dir = (int64_t)hs.dir_nodes.size();
  std::vector<int32_t> inode(h->nI_tot), gnode(h->nG_tot), csub(h->nC_tot), ccdof(h->nC_tot);
  std::vector<double> gw(h->nG_tot);
  for (int s = 0; s < S; ++s) {
    std::copy(hs.sub_I[s].begin(), hs.sub_I[s].end(), inode.begin() + ioff[s]);
    for (size_t l = 0; l < hs.sub_G[s].size(); ++l) {
      gnode[goff[s] + l] = hs.sub_G[s][l];
      gw[goff[s] + l] = 1.0 / hs.kappa[hs.sub_G[s][l]];
    }
    for (size_t r = 0; r < hs.sub_globs[s].size(); ++r) {
      csub[coff[s] + r] = s;
      ccdof[coff[s] + r] = hs.sub_globs[s][r];
    }
  }
  // sparse coarse solve: the coarse dofs are numbered in elimination order on
  // the device (r_c, u_c and the factor then share one order, and the sweeps
  // read and write contiguous runs); cperm maps a glob to that number
  std::vector<int32_t> cperm;
  if (hs.n_c && !hs.coarse_dense && !hs.coarse_cg) {
    coarse_renumber(hs.cfac, cperm);
    for (auto& c : ccdof) c = cperm[c];
  }
  // sparse local solver: each subdomain's compact interior positions are
  // numbered in the elimination order of its factor (the interior sweeps
  // then read and write contiguous runs); iperm[s][local] = position
  std::vector<std::vector<int32_t>> iperm(hs.sparse_local ? S : 0), iinv(hs.sparse_local ? S : 0);
  if (hs.sparse_local) {
    for (int s = 0; s < S; ++s) {
      coarse_renumber(hs.ifac[s], iperm[s]);
      iinv[s].assign(iperm[s].size(), 0);
      for (size_t l = 0; l < iperm[s].size(); ++l) {
        iinv[s][iperm[s][l]] = (int32_t)l;
        inode[ioff[s] + iperm[s][l]] = hs.sub_I[s][l];
      }
    }
  }
  // A_GI with global compact interior columns; A_IG with node-id columns
  std::vector<int32_t> agi_ptr(h->nG_tot + 1, 0), agi_col, aig_ptr(h->nI_tot + 1, 0), aig_col;
  std::vector<double> agi_val, aig_val;
  for (int s = 0; s < S; ++s) {
    const int nG = (int)hs.sub_G[s].size(), nI = (int)hs.sub_I[s].size();
    for (int r = 0; r < nG; ++r) {
      for (int j = hs.agi_ptr[s][r]; j < hs.agi_ptr[s][r + 1]; ++j) {
        const int32_t c = hs.agi_col[s][j];
        agi_col.push_back(ioff[s] + (hs.sparse_local ? iperm[s][c] : c));
        agi_val.push_back(hs.agi_val[s][j]);
      }
      agi_ptr[goff[s] + r + 1] = (int32_t)agi_col.size();
    }
    for (int q = 0; q < nI; ++q) {
      const int r = hs.sparse_local ? iinv[s][q] : q;
      for (int j = hs.aig_ptr[s][r]; j < hs.aig_ptr[s][r + 1]; ++j) {
        aig_col.push_back(hs.sub_G[s][hs.aig_col[s][j]]);
        aig_val.push_back(hs.aig_val[s][j]);
      }
      aig_ptr[ioff[s] + q + 1] = (int32_t)aig_col.size();
    }
  }
  // Phi_G^T (n_c x n_G per subdomain: coarse residual) and Phi_G (n_G x n_c:
  // prolongation), float64, as batched operators of the streamed GEMV
  std::vector<int> nGv(S), ncv(S);
  for (int s = 0; s < S; ++s) { nGv[s] = (int)hs.sub_G[s].size(); ncv[s] = (int)hs.sub_globs[s].size(); }
  std::vector<int64_t> ptoff;
  std::vector<int32_t> ptld;
  const int phi_eb = elem_bytes(h->phi_prec);
  std::vector<double> phit = pack_rect(hs.Phi, ncv, nGv, true, phi_eb, ptoff, ptld);
  auto itPT = make_rect_items(ptoff, ptld, ncv, nGv, goff, coff, 128);
  h->n_wi_PT = (int)itPT.size();
  h->max_ld_PT = ptld.empty() ? 0 : *std::max_element(ptld.begin(), ptld.end());
  // coarse gather map: coarse dof -> local constraint positions
  std::vector<int32_t> cg_ptr(hs.n_c + 1, 0), cg_idx(h->nC_tot);
  for (int64_t j = 0; j < h->nC_tot; ++j) cg_ptr[ccdof[j] + 1]++;
  for (int64_t c = 0; c < hs.n_c; ++c) cg_ptr[c + 1] += cg_ptr[c];
  {
    std::vector<int32_t> fill(cg_ptr.begin(), cg_ptr.end() - 1);
    for (int64_t j = 0; j < h->nC_tot; ++j) cg_idx[fill[ccdof[j]]++] = (int32_t)j;
  }
  // unique interface nodes and their copies
  std::vector<int32_t> gu_node;
  std::vector<int32_t> node2gu(hs.n_nodes, -1);
  for (int64_t n = 0; n < hs.n_nodes; ++n)
    if (hs.kappa[n] >= 2) { node2gu[n] = (int32_t)gu_node.size(); gu_node.push_back((int32_t)n); }
  h->n_gu = (int64_t)gu_node.size();
  std::vector<int32_t> gu_ptr(h->n_gu + 1, 0), gu_copy(h->nG_tot);
  for (int64_t q = 0; q < h->nG_tot; ++q) gu_ptr[node2gu[gnode[q]] + 1]++;
  for (int64_t u = 0; u < h->n_gu; ++u) gu_ptr[u + 1] += gu_ptr[u];
  {
    std::vector<int32_t> fill(gu_ptr.begin(), gu_ptr.end() - 1);
    for (int64_t q = 0; q < h->nG_tot; ++q) gu_copy[fill[node2gu[gnode[q]]]++] = (int32_t)q;
  }
  // ---- operator arenas ----------------------------------------------------------
  std::vector<int> dI(S), dG(S);
  for (int s = 0; s < S; ++s) { dI[s] = (int)hs.sub_I[s].size(); dG[s] = (int)hs.sub_G[s].size(); }
  // the dense interior operators (none with the sparse local solver)
  const std::vector<int> dIop = hs.sparse_local ? std::vector<int>(S, 0) : dI;
  std::vector<int64_t> offI, offG;
  std::vector<int32_t> ldI, ldG;
  const int prec = h->precision;
  size_t arena_bytes = 0;
  auto up_arena = [&](const std::vector<std::vector<double>>& ops, const std::vector<int>& dims,
                      std::vector<int64_t>& off, std::vector<int32_t>& ld, void** dst) -> cudaError_t {
    if (prec == BDDC_PREC_FP64) {
      auto a = pack_arena<double>(ops, dims, off, ld, cvt_d);
      arena_bytes += a.size() * sizeof(double);
      return upload(h, reinterpret_cast<double**>(dst), a);
    } else if (prec == BDDC_PREC_FP32) {
      auto a = pack_arena<float>(ops, dims, off, ld, cvt_f);
      arena_bytes += a.size() * sizeof(float);
      return upload(h, reinterpret_cast<float**>(dst), a);
    }
    auto a = pack_arena<__nv_bfloat16>(ops, dims, off, ld, cvt_b);
    arena_bytes += a.size() * sizeof(__nv_bfloat16);
    return upload(h, reinterpret_cast<__nv_bfloat16**>(dst), a);
  };
  int64_t opbytes_I = 0, opbytes_G = 0;
  if (h->use_tc) {
    // tensor-core path: operators in the MMA tile layout, no row-major copy
    auto up_tc = [&](auto tag, const std::vector<std::vector<double>>& ops, const std::vector<int>& dims,
                     const std::vector<int32_t>& xo, void** arena, TcUnit** units, int* n_units, int32_t** sl,
                     int64_t* n_sl, int32_t** opi, int64_t* cols, int64_t* bytes, int* maxg) -> int {
      using T = decltype(tag);
      TcPacked<T> pk;
      tc_pack_host<T>(ops, dims, xo, pk);
      *bytes = (int64_t)(pk.arena.size() * sizeof(T));
      arena_bytes += pk.arena.size() * sizeof(T);
      *n_units = (int)pk.units.size();
      *n_sl = (int64_t)pk.slice_op.size();
      *cols = pk.cols_total;
      *maxg = pk.max_g;
      CUDA_TRY(upload(h, reinterpret_cast<T**>(arena), pk.arena));
      CUDA_TRY(upload(h, units, pk.units));
      CUDA_TRY(upload(h, sl, pk.slice_op));
      CUDA_TRY(upload(h, opi, pk.opinfo));
      return BDDC_OK;
    };
    int rc2;
    if (prec == BDDC_PREC_BF16) {
      if ((rc2 = up_tc(__nv_bfloat16{}, hs.AIIinv, dIop, ioff, &h->d_aii, &h->d_tcu_I, &h->n_tcu_I, &h->d_tcs_I,
                       &h->n_tcs_I, &h->d_tcop_I, &h->tcB_cols_I, &opbytes_I, &h->tc_maxg_I)) != BDDC_OK)
        return rc2;
      if ((rc2 = up_tc(__nv_bfloat16{}, hs.Kgg, dG, goff, &h->d_kgg, &h->d_tcu_G, &h->n_tcu_G, &h->d_tcs_G,
                       &h->n_tcs_G, &h->d_tcop_G, &h->tcB_cols_G, &opbytes_G, &h->tc_maxg_G)) != BDDC_OK)
        return rc2;
    } else {
      if ((rc2 = up_tc(float{}, hs.AIIinv, dIop, ioff, &h->d_aii, &h->d_tcu_I, &h->n_tcu_I, &h->d_tcs_I, &h->n_tcs_I,
                       &h->d_tcop_I, &h->tcB_cols_I, &opbytes_I, &h->tc_maxg_I)) != BDDC_OK)
        return rc2;
      if ((rc2 = up_tc(float{}, hs.Kgg, dG, goff, &h->d_kgg, &h->d_tcu_G, &h->n_tcu_G, &h->d_tcs_G, &h->n_tcs_G,
                       &h->d_tcop_G, &h->tcB_cols_G, &opbytes_G, &h->tc_maxg_G)) != BDDC_OK)
        return rc2;
    }
    const size_t bbytes = tc_operand_bytes(prec, std::max(h->tcB_cols_I, h->tcB_cols_G), h->nrhs_max);
    void* pB = nullptr;
    CUDA_TRY(cudaMalloc(&pB, bbytes));
    h->allocations.push_back(pB);
    h->d_tcB = pB;
    h->use_tma = false;
  } else if (!h->full_operators && h->nrhs_max == 1 && (prec == BDDC_PREC_FP32 || prec == BDDC_PREC_BF16) &&
             sgemv_tma_supported(prec, std::max(dIop.empty() ? 0 : *std::max_element(dIop.begin(), dIop.end()),
                                                dG.empty() ? 0 : *std::max_element(dG.begin(), dG.end())))) {
    // symmetric operators, one right-hand side: lower triangles, one work
    // item per operator (largest first)
    auto up_sym = [&](const std::vector<std::vector<double>>& ops, const std::vector<int>& dims,
                      const std::vector<int32_t>& voff, void** arena, WorkItem** items, int* n_items, int* max_n,
                      int64_t* bytes) -> cudaError_t {
      std::vector<int64_t> off;
      cudaError_t e;
      if (prec == BDDC_PREC_FP32) {
        auto a = pack_lower<float>(ops, dims, prec, off, cvt_f);
        arena_bytes += a.size() * sizeof(float);
        e = upload(h, reinterpret_cast<float**>(arena), a);
      } else {
        auto a = pack_lower<__nv_bfloat16>(ops, dims, prec, off, cvt_b);
        arena_bytes += a.size() * sizeof(__nv_bfloat16);
        e = upload(h, reinterpret_cast<__nv_bfloat16**>(arena), a);
      }
      if (e != cudaSuccess) return e;
      std::vector<WorkItem> it;
      *bytes = 0;
      *max_n = 0;
      for (size_t s = 0; s < dims.size(); ++s) {
        if (dims[s] == 0) continue;
        it.push_back(WorkItem{off[s], padded_ld(dims[s], elem_bytes(prec)), dims[s], 0, dims[s], voff[s], voff[s]});
        *bytes += sym_packed_elems(prec, dims[s]) * elem_bytes(prec);
        *max_n = std::max(*max_n, dims[s]);
      }
      std::stable_sort(it.begin(), it.end(), [](const WorkItem& a, const WorkItem& b) { return a.ncols > b.ncols; });
      *n_items = (int)it.size();
      return upload(h, items, it);
    };
    CUDA_TRY(up_sym(hs.AIIinv, dIop, ioff, reinterpret_cast<void**>(&h->d_aii), &h->d_wsy_I, &h->n_wsy_I,
                    &h->max_n_I, &opbytes_I));
    CUDA_TRY(up_sym(hs.Kgg, dG, goff, reinterpret_cast<void**>(&h->d_kgg), &h->d_wsy_G, &h->n_wsy_G, &h->max_n_G,
                    &opbytes_G));
    h->use_sym = true;
    h->use_tma = true;
  } else {
    CUDA_TRY(up_arena(hs.AIIinv, dIop, offI, ldI, &h->d_aii));
    CUDA_TRY(up_arena(hs.Kgg, dG, offG, ldG, &h->d_kgg));
    const int tile = 64;
    auto itI = make_items(offI, ldI, dIop, ioff, tile);
    auto itG = make_items(offG, ldG, dG, goff, tile);
    h->n_wi_I = (int)itI.size();
    h->n_wi_G = (int)itG.size();
    h->max_cols_I = ldI.empty() ? 0 : *std::max_element(ldI.begin(), ldI.end());
    h->max_cols_G = ldG.empty() ? 0 : *std::max_element(ldG.begin(), ldG.end());
    CUDA_TRY(upload(h, &h->d_wi_I, itI));
    CUDA_TRY(upload(h, &h->d_wi_G, itG));
    h->use_tma = bgemv_tma_supported(prec, h->max_cols_I) && bgemv_tma_supported(prec, h->max_cols_G);
    // work lists of the streamed GEMV for row tiles of 64, 128 and 256 rows
    // (the autotuner picks one per operator family; 128 by default)
    for (int c = 0; c < 3; ++c) {
      const int ttile = 64 << c;
      auto tI = make_items(offI, ldI, dIop, ioff, ttile);
      auto tG = make_items(offG, ldG, dG, goff, ttile);
      h->n_wtx_I[c] = (int)tI.size();
      h->n_wtx_G[c] = (int)tG.size();
      if (!items_aligned(tI, elem_bytes(prec)) || !items_aligned(tG, elem_bytes(prec)))
        return fail(BDDC_ERR_INVALID_ARG, "internal: local operator rows not 16-byte aligned");
      CUDA_TRY(upload(h, &h->d_wtx_I[c], tI));
      CUDA_TRY(upload(h, &h->d_wtx_G[c], tG));
    }
    for (int s = 0; s < S; ++s) {
      opbytes_I += (int64_t)dIop[s] * ldI[s] * elem_bytes(prec);
      opbytes_G += (int64_t)dG[s] * ldG[s] * elem_bytes(prec);
    }
  }
  h->coarse_dense = hs.coarse_dense;
  h->coarse_cg = hs.coarse_cg;
  if (hs.n_c && hs.coarse_cg) {
    // A_c in CSR (both triangles, glob order) for the coarse CG; one block
    // per SM (cooperative launch)
    std::vector<int32_t> acp(hs.Ac_ptr.begin(), hs.Ac_ptr.end());
    CUDA_TRY(upload(h, &h->d_acp, acp));
    CUDA_TRY(upload(h, &h->d_acc, hs.Ac_col));
    CUDA_TRY(upload(h, &h->d_acv, hs.Ac_val));
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&h->c_sms, cudaDevAttrMultiProcessorCount, dev));
    h->c_nnz = (int64_t)hs.Ac_val.size();
    CUDA_TRY(build_coarse_cg_device(h));
    in_coarse_bytes = h->c_nnz * 12 + (hs.n_c + 1) * 4;
    coarse_read_1rhs = in_coarse_bytes;   // one product with A_c (per coarse CG iteration)
  } else if (hs.n_c && hs.coarse_dense) {
    // A_c^-1, float64, stored as column panels of kPanel columns (each an
    // n_c x width row-major block, blocks aligned to 256 bytes); the panels'
    // partial products are summed by a separate kernel
    std::vector<WorkItem> itC;
    const int kPanel = 512;
    const int nc = (int)hs.n_c;
    h->ldc = kPanel;
    h->n_cpanels = (nc + kPanel - 1) / kPanel;
    std::vector<int64_t> poff(h->n_cpanels);
    std::vector<int32_t> pw(h->n_cpanels), pld(h->n_cpanels);
    int64_t cur = 0;
    for (int p = 0; p < h->n_cpanels; ++p) {
      cur = (cur + 31) / 32 * 32;
      poff[p] = cur;
      pw[p] = std::min(kPanel, nc - p * kPanel);
      pld[p] = padded_ld(pw[p], 8);
      cur += (int64_t)nc * pld[p];
    }
    std::vector<double> ac((size_t)cur, 0.0);
    for (int p = 0; p < h->n_cpanels; ++p)
      for (int r = 0; r < nc; ++r)
        std::memcpy(&ac[poff[p] + (int64_t)r * pld[p]], &hs.Acinv[(size_t)r * nc + (size_t)p * kPanel],
                    sizeof(double) * pw[p]);
    std::vector<double>().swap(hs.Acinv);
    CUDA_TRY(upload(h, &h->d_acinv, ac));
    in_coarse_bytes = cur * 8;
    coarse_read_1rhs = in_coarse_bytes;
    h->c_nnz = cur;
    const int ctile = 128;
    for (int p = 0; p < h->n_cpanels; ++p)
      for (int r0 = 0; r0 < nc; r0 += ctile)
        itC.push_back(WorkItem{poff[p], pld[p], pw[p], r0, std::min(ctile, nc - r0), p * kPanel, p * nc});
    h->n_wi_C = (int)itC.size();
    if (!items_aligned(itC, 8)) return fail(BDDC_ERR_INVALID_ARG, "internal: coarse panels not 16-byte aligned");
    CUDA_TRY(upload(h, &h->d_wi_C, itC));
  } else if (hs.n_c) {
    // sparse Cholesky factorisation of A_c: supernode matrices and level lists
    CUDA_TRY(build_coarse_device(h, hs.cfac));
    in_coarse_bytes = h->c_nnz * 8 + h->cs.g_entries * 12;
    coarse_read_1rhs = h->cs.g_entries * 12;
  }
  // ---- sparse local solver: the interior factors as one forest ----------------------
  h->sparse_local = hs.sparse_local;
  int64_t ifac_entries = 0;
  if (hs.sparse_local && h->nI_tot > 0) {
    CoarseFactor forest;
    merge_forest(hs.ifac, ioff, forest);
    std::vector<CoarseFactor>().swap(hs.ifac);
    ifac_entries = forest.nnz;
    // the mixed forms sweep in float32 (an inexact interior solve inside
    // flexible PCG, as the low-precision dense operators are); FP64 in float64
    const bool c32 = h->precision != BDDC_PREC_FP64;
    CUDA_TRY(build_sweeps(h, forest, h->is, h->nrhs_max > 1, 0, c32 ? kSweepLevel : kSweepBlock, c32));
    // one interior solve at one column reads its coefficients once
    opbytes_I = sweep_read_1col(h->is);
    arena_bytes += (size_t)(h->is.g_entries * 12 + ((h->is.multi || h->is.block_form) ? h->is.nnz * 8 : 0));
  }
  // ---- index arrays -----------------------------------------------------------------
  std::vector<double> sigma(P->elem_sigma, P->elem_sigma + hs.n_elems);
  CUDA_TRY(upload(h, &h->d_sigma, sigma));
  CUDA_TRY(upload(h, &h->d_dnode, hs.dir_nodes));
  CUDA_TRY(upload(h, &h->d_inode, inode));
  CUDA_TRY(upload(h, &h->d_gnode, gnode));
  CUDA_TRY(upload(h, &h->d_gw, gw));
  CUDA_TRY(upload(h, &h->d_agi_ptr, agi_ptr));
  CUDA_TRY(upload(h, &h->d_agi_col, agi_col));
  CUDA_TRY(upload(h, &h->d_agi_val, agi_val));
  CUDA_TRY(upload(h, &h->d_aig_ptr, aig_ptr));
  CUDA_TRY(upload(h, &h->d_aig_col, aig_col));
  CUDA_TRY(upload(h, &h->d_aig_val, aig_val));
  if (h->phi_prec == BDDC_PREC_FP32) {
    std::vector<float> f32(phit.begin(), phit.end());
    CUDA_TRY(upload(h, reinterpret_cast<float**>(&h->d_phit), f32));
  } else {
    CUDA_TRY(upload(h, reinterpret_cast<double**>(&h->d_phit), phit));
  }
  if (!items_aligned(itPT, phi_eb)) return fail(BDDC_ERR_INVALID_ARG, "internal: Phi rows not 16-byte aligned");
  CUDA_TRY(upload(h, &h->d_wi_PT, itPT));
  CUDA_TRY(upload(h, &h->d_pt_off, ptoff));
  CUDA_TRY(upload(h, &h->d_pt_ld, ptld));
  CUDA_TRY(upload(h, &h->d_sub_goff, goff));
  CUDA_TRY(upload(h, &h->d_sub_coff, coff));
  CUDA_TRY(upload(h, &h->d_csub, csub));
  CUDA_TRY(upload(h, &h->d_ccdof, ccdof));
  if (!cperm.empty()) CUDA_TRY(upload(h, &h->d_cperm, cperm));
  CUDA_TRY(upload(h, &h->d_cg_ptr, cg_ptr));
  CUDA_TRY(upload(h, &h->d_cg_idx, cg_idx));
  CUDA_TRY(upload(h, &h->d_gu_node, gu_node));
  CUDA_TRY(upload(h, &h->d_gu_ptr, gu_ptr));
  CUDA_TRY(upload(h, &h->d_gu_copy, gu_copy));

  // ---- workspace ---------------------------------------------------------------------
  const int64_t R = h->nrhs_max;
  CUDA_TRY(dev_alloc(h, &h->w.rI, h->nI_tot * R));
  CUDA_TRY(dev_alloc(h, &h->w.tI, h->nI_tot * R));
  CUDA_TRY(dev_alloc(h, &h->w.bI, h->nI_tot * R));
  if (h->sparse_local) {
    CUDA_TRY(dev_alloc(h, &h->w.ir, h->nI_tot * R));
    CUDA_TRY(dev_alloc(h, &h->w.iy, h->nI_tot * R));
  }
  CUDA_TRY(dev_alloc(h, &h->w.yG, h->nG_tot * R));
  CUDA_TRY(dev_alloc(h, &h->w.zG, h->nG_tot * R));
  CUDA_TRY(dev_alloc(h, &h->w.eG, h->nG_tot * R));
  CUDA_TRY(dev_alloc(h, &h->w.g, h->nC_tot * R));
  CUDA_TRY(dev_alloc(h, &h->w.rc, h->n_c * R));
  CUDA_TRY(dev_alloc(h, &h->w.uc, h->n_c * R));
  if (h->coarse_dense) {
    CUDA_TRY(dev_alloc(h, &h->w.cpart, (int64_t)std::max(1, h->n_cpanels) * h->n_c * R));
  } else {
    CUDA_TRY(dev_alloc(h, &h->w.cr, h->n_c * R));
    CUDA_TRY(dev_alloc(h, &h->w.cy, h->n_c * R));
  }
  if (h->coarse_cg) {
    CUDA_TRY(dev_alloc(h, &h->w.cq, h->n_c * R));
    CUDA_TRY(dev_alloc(h, &h->d_cgpart, (size_t)std::max(1, h->c_sms) * 2 * R));
    CUDA_TRY(dev_alloc(h, &h->d_cgiters, (size_t)R));
    CUDA_TRY(cudaMemset(h->d_cgiters, 0, sizeof(int32_t) * R));
  }
  CUDA_TRY(cudaMemset(h->w.rc, 0, std::max<int64_t>(1, h->n_c * R) * sizeof(double)));
  CUDA_TRY(cudaMemset(h->w.uc, 0, std::max<int64_t>(1, h->n_c * R) * sizeof(double)));
  const int64_t NV = h->n_nodes * R;
  CUDA_TRY(dev_alloc(h, &h->p_r, NV));
  CUDA_TRY(dev_alloc(h, &h->p_z, NV));
  CUDA_TRY(dev_alloc(h, &h->p_zold, NV));
  CUDA_TRY(dev_alloc(h, &h->p_p, NV));
  CUDA_TRY(dev_alloc(h, &h->p_q, NV));
  CUDA_TRY(dev_alloc(h, &h->s_b, NV));
  CUDA_TRY(dev_alloc(h, &h->s_x, NV));
  h->n_red_blocks = kRedBlocks;
  CUDA_TRY(dev_alloc(h, &h->d_partials, (size_t)kRedBlocks * 3 * R));
  CUDA_TRY(dev_alloc(h, &h->d_counter, 1));
  CUDA_TRY(cudaMemset(h->d_counter, 0, sizeof(unsigned int)));
  CUDA_TRY(dev_alloc(h, &h->d_stencil,
                     (size_t)stencil_points(h->dim) * (h->n_nodes + 2 * stencil_guard(h->dim, h->ne))));
  CUDA_TRY(launch_build_stencil(h, nullptr));
  CUDA_TRY(dev_alloc(h, &h->d_scal, (size_t)S_COUNT * R));
  CUDA_TRY(dev_alloc(h, &h->d_iscal, (size_t)I_COUNT * R + kGlobalFlags));
  CUDA_TRY(cudaMemset(h->d_scal, 0, sizeof(double) * S_COUNT * R));
  CUDA_TRY(cudaMemset(h->d_iscal, 0, sizeof(int32_t) * (I_COUNT * R + kGlobalFlags)));
  CUDA_TRY(cudaMallocHost(&h->h_flags, sizeof(int32_t) * (I_COUNT * R + kGlobalFlags)));
  h->d_err = h->d_iscal + I_COUNT * R + 2;
  if (h->hist_cap > 0) CUDA_TRY(dev_alloc(h, &h->d_hist, (size_t)3 * (h->hist_cap + 1) * R));
  // ---- info ------------------------------------------------------------------------
  bddc_info_t& in = h->info;
  in.n_nodes = hs.n_nodes;
  in.n_free = hs.n_nodes - h->n_dir;
  in.n_interior = h->nI_tot;
  in.n_interface_nodes = h->n_gu;
  in.n_sub = S;
  in.n_c = hs.n_c;
  for (int k : hs.glob_kind) {
    if (k == BDDC_CORNERS) in.n_corners++;
    else if (k == BDDC_EDGES) in.n_edges++;
    else in.n_faces++;
  }
  for (int s = 0; s < S; ++s) {
    const int64_t nI = dI[s], nG = dG[s], nc = (int64_t)hs.sub_globs[s].size();
    in.sum_ni += nI + nG;
    in.sum_nI2 += nI * nI;
    in.sum_nG2 += nG * nG;
    in.sum_nG_nc += nG * nc;
    in.max_ni = std::max(in.max_ni, nI + nG);
  }
  in.operator_bytes = (int64_t)arena_bytes;
  in.coarse_bytes = in_coarse_bytes;
  // compulsory HBM bytes of one apply (nrhs = 1): operators as stored (A_II^-1
  // read twice), Phi rows twice, the coarse inverse (or the gather form of the
  // sparse factor: coefficients and operand indices) once, the sparse
  // couplings, the input r and the output z.
  int64_t ops = 0;
  in.interior_op_bytes = opbytes_I;
  in.local_solver = h->sparse_local ? BDDC_LOCAL_SPARSE : BDDC_LOCAL_DENSE;
  in.interior_levels = h->sparse_local ? h->is.levels : 0;
  in.interior_factor_entries = ifac_entries;
  in.interface_op_bytes = opbytes_G;
  in.tensor_cores = h->use_tc ? 1 : 0;
  in.symmetric_operators = h->use_sym ? 1 : 0;
  in.n_interface_copies = h->nG_tot;
  in.coarse_factor_entries = h->c_nnz;
  in.coarse_update_total = h->cs.update_total;
  in.coarse_levels = h->coarse_dense || h->coarse_cg ? 0 : h->cs.levels;
  ops = 2 * in.interior_op_bytes + in.interface_op_bytes;
  in.phi_precision = h->phi_prec;
  in.apply_bytes_1rhs = ops + 2 * (int64_t)elem_bytes(h->phi_prec) * in.sum_nG_nc + coarse_read_1rhs +
                        (int64_t)(agi_val.size() + aig_val.size()) * 12 + 8 * (in.n_free + hs.n_nodes);
  return BDDC_OK;
}

// Drop the captured PCG graphs (they hold launch arguments that changed).
void drop_graphs(bddc_handle_t h) {
  if (h->iter_graph) {
    cudaGraphExecDestroy(h->iter_graph);
    h->iter_graph = nullptr;
  }
  if (h->solve_graph) {
    cudaGraphExecDestroy(h->solve_graph);
    h->solve_graph = nullptr;
  }
}

int check_handle(bddc_handle_t h, int nrhs) {
  if (!h) return fail(BDDC_ERR_INVALID_ARG, "null handle");
  if (nrhs < 1 || nrhs > h->nrhs_max)
    return fail(BDDC_ERR_INVALID_ARG, "nrhs " + std::to_string(nrhs) + " outside [1, nrhs_max=" +
                                          std::to_string(h->nrhs_max) + "]");
  return BDDC_OK;
}

#define ENTER_DEVICE(dev)                                                                   \
  DeviceGuard device_guard_(dev);                                                           \
  if (!device_guard_.ok) return fail(BDDC_ERR_CUDA, "could not make the handle's device current")

}  // namespace

int bddc::set_last_error(int code, const std::string& msg) { return fail(code, msg); }

extern "C" {

const char* bddc_strerror(int status) {
  switch (status) {
    case BDDC_OK: return "ok";
    case BDDC_NOT_CONVERGED: return "PCG did not reach rtol within maxit iterations";
    case BDDC_ERR_INVALID_ARG: return "invalid argument";
    case BDDC_ERR_OOM: return "out of memory";
    case BDDC_ERR_CUDA: return "CUDA runtime error";
    case BDDC_ERR_SINGULAR: return "singular local or coarse matrix in setup";
    case BDDC_ERR_TIMEOUT: return "bounded device wait timed out";
    case BDDC_ERR_BREAKDOWN: return "PCG breakdown (p^T A p <= 0 or non-finite)";
    case BDDC_ERR_NO_DEVICE: return "no usable CUDA device";
    default: return "unknown status";
  }
}

const char* bddc_last_error(void) { return g_last_error.c_str(); }

void bddc_destroy(bddc_handle_t h) {
  if (!h) return;
  DeviceGuard device_guard_(h->device);
  if (h->iter_graph) cudaGraphExecDestroy(h->iter_graph);
  if (h->solve_graph) cudaGraphExecDestroy(h->solve_graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->body_stream) cudaStreamDestroy(h->body_stream);
  for (int a = 0; a < 2; ++a) {
    if (h->aux_stream[a]) cudaStreamDestroy(h->aux_stream[a]);
    if (h->ev_fork[a]) cudaEventDestroy(h->ev_fork[a]);
    if (h->ev_join[a]) cudaEventDestroy(h->ev_join[a]);
  }
  for (void* p : h->allocations) cudaFree(p);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  delete h;
}

int bddc_setup(const bddc_problem_t* P, const bddc_options_t* O, bddc_handle_t* out) {
  g_last_error.clear();
  if (!P || !O || !out) return fail(BDDC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const auto t0 = std::chrono::steady_clock::now();
  {
    std::string verr;
    int vrc = validate_problem(P, O, verr);
    if (vrc != BDDC_OK) return fail(vrc, verr);
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(BDDC_ERR_NO_DEVICE, "no CUDA device");
  if (O->device < 0 || O->device >= ndev) return fail(BDDC_ERR_INVALID_ARG, "device ordinal out of range");
  ENTER_DEVICE(O->device);
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, O->device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(BDDC_ERR_NO_DEVICE, std::string("device is not sm_103: ") + prop.name);

  HostSetup hs;
  std::string err;
  int rc = host_setup(P, O, hs, err);
  if (rc != BDDC_OK) return fail(rc, err);

  bddc_handle_s* h = new (std::nothrow) bddc_handle_s();
  if (!h) return fail(BDDC_ERR_OOM, "handle allocation");
  h->dim = P->dim; h->ne = P->ne; h->n1 = P->ne + 1; h->n_sub = P->n_sub;
  h->precision = effective_precision(O); h->nrhs_max = O->nrhs_max; h->device = O->device;
  h->use_graph = O->no_graph == 0;
  h->phi_prec = (O->precision == BDDC_PREC_FP64 || O->phi_fp64) ? BDDC_PREC_FP64 : BDDC_PREC_FP32;
  h->use_tc = tc_enabled(O);
  h->g_blocks = O->coarse_blocks;
  h->full_operators = O->full_operators != 0;
  h->hist_cap = O->history;
  h->cg_maxit = O->coarse_cg_maxit > 0 ? O->coarse_cg_maxit : 2000;
  h->cg_rtol = O->coarse_cg_rtol > 0.0 ? O->coarse_cg_rtol : 1e-10;
  h->n_nodes = hs.n_nodes; h->n_elems = hs.n_elems; h->h = hs.h;
  rc = build_device(h, hs, P);
  if (rc != BDDC_OK) {
    bddc_destroy(h);
    return rc;
  }
  cudaError_t e = cudaDeviceSynchronize();
  for (int a = 0; a < 2 && e == cudaSuccess; ++a) {
    e = cudaStreamCreateWithFlags(&h->aux_stream[a], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork[a], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join[a], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    bddc_destroy(h);
    return fail(BDDC_ERR_CUDA, cudaGetErrorString(e));
  }
  h->info.precision = h->precision;
  h->info.error_subdomain = -1;
  h->info.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return BDDC_OK;
}

int bddc_setup_inspect(const bddc_problem_t* P, const bddc_options_t* O, int32_t numerics, bddc_info_t* info,
                       double* Ac, int64_t Ac_capacity) {
  g_last_error.clear();
  std::string err;
  int rc = validate_problem(P, O, err);
  if (rc != BDDC_OK) return fail(rc, err);
  HostSetup hs;
  rc = host_setup(P, O, hs, err, /*invert_coarse=*/false, /*numerics=*/numerics != 0);
  if (rc != BDDC_OK) return fail(rc, err);
  if (info) {
    *info = bddc_info_t{};
    info->n_nodes = hs.n_nodes;
    info->n_free = hs.n_nodes - (int64_t)hs.dir_nodes.size();
    info->n_sub = hs.n_sub;
    info->n_c = hs.n_c;
    for (int k : hs.glob_kind) {
      if (k == BDDC_CORNERS) info->n_corners++;
      else if (k == BDDC_EDGES) info->n_edges++;
      else info->n_faces++;
    }
    for (int s = 0; s < hs.n_sub; ++s) {
      const int64_t nI = (int64_t)hs.sub_I[s].size(), nG = (int64_t)hs.sub_G[s].size();
      info->n_interior += nI;
      info->sum_ni += nI + nG;
      info->sum_nI2 += nI * nI;
      info->sum_nG2 += nG * nG;
      info->sum_nG_nc += nG * (int64_t)hs.sub_globs[s].size();
      info->max_ni = std::max(info->max_ni, nI + nG);
    }
    for (int64_t n = 0; n < hs.n_nodes; ++n) info->n_interface_nodes += hs.kappa[n] >= 2;
    info->error_subdomain = -1;
    info->precision = effective_precision(O);
    info->phi_precision =
        (O->precision == BDDC_PREC_FP64 || O->phi_fp64) ? BDDC_PREC_FP64 : BDDC_PREC_FP32;
    info->tensor_cores = tc_enabled(O) ? 1 : 0;
  }
  if (Ac && numerics) {
    if (hs.n_c * hs.n_c > Ac_capacity) return fail(BDDC_ERR_INVALID_ARG, "Ac capacity too small");
    std::fill(Ac, Ac + hs.n_c * hs.n_c, 0.0);
    for (int64_t r = 0; r < hs.n_c; ++r)
      for (int64_t j = hs.Ac_ptr[r]; j < hs.Ac_ptr[r + 1]; ++j) Ac[r * hs.n_c + hs.Ac_col[j]] = hs.Ac_val[j];
  }
  return BDDC_OK;
}

int bddc_query(bddc_handle_t h, bddc_info_t* info) {
  if (!h || !info) return fail(BDDC_ERR_INVALID_ARG, "null argument");
  h->info.kernel_launches = h->launches;
  h->info.solve_graph = h->use_graph && !h->solve_graph_unsupported ? 1 : 0;
  ENTER_DEVICE(h->device);
  CUDA_TRY(cudaMemcpy(&h->info.device_error, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  h->info.coarse_cg_iters = 0;
  if (h->d_cgiters) {
    std::vector<int32_t> it(h->nrhs_max);
    CUDA_TRY(cudaMemcpy(it.data(), h->d_cgiters, sizeof(int32_t) * h->nrhs_max, cudaMemcpyDeviceToHost));
    h->info.coarse_cg_iters = *std::max_element(it.begin(), it.end());
  }
  *info = h->info;
  return BDDC_OK;
}

int bddc_apply(bddc_handle_t h, const double* r, double* z, int32_t nrhs, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!r || !z || r == z) return fail(BDDC_ERR_INVALID_ARG, "r and z must be distinct device pointers");
  CUDA_TRY(launch_apply(h, r, z, nrhs, static_cast<cudaStream_t>(stream)));
  return BDDC_OK;
}

int bddc_matvec(bddc_handle_t h, const double* x, double* y, int32_t nrhs, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!x || !y || x == y) return fail(BDDC_ERR_INVALID_ARG, "x and y must be distinct device pointers");
  CUDA_TRY(launch_spmv(h, x, y, nrhs, -1, 0.0, 0, static_cast<cudaStream_t>(stream)));
  return BDDC_OK;
}

int bddc_rhs(bddc_handle_t h, const double* f, double* b, int32_t nrhs, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!f || !b || f == b) return fail(BDDC_ERR_INVALID_ARG, "f and b must be distinct device pointers");
  CUDA_TRY(launch_rhs(h, f, b, nrhs, static_cast<cudaStream_t>(stream)));
  return BDDC_OK;
}

int bddc_elem_grad(bddc_handle_t h, const double* u, const double* lambda, double* g, int32_t nrhs, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!u || !lambda || !g) return fail(BDDC_ERR_INVALID_ARG, "u, lambda and g must be device pointers");
  CUDA_TRY(launch_elem_grad(h, u, lambda, g, nrhs, static_cast<cudaStream_t>(stream)));
  return BDDC_OK;
}

int bddc_coarse_vectors(bddc_handle_t h, double* rc_out, double* uc_out, int32_t nrhs, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)h->n_c * nrhs * sizeof(double);
  if (bytes == 0) return BDDC_OK;
  // in glob order (the sparse coarse solve numbers the coarse dofs in its
  // elimination order on the device)
  if (h->d_cperm) {
    if (rc_out) CUDA_TRY(launch_gather_rows(h->n_c, nrhs, h->d_cperm, h->w.rc, rc_out, st));
    if (uc_out) CUDA_TRY(launch_gather_rows(h->n_c, nrhs, h->d_cperm, h->w.uc, uc_out, st));
    return BDDC_OK;
  }
  if (rc_out) CUDA_TRY(cudaMemcpyAsync(rc_out, h->w.rc, bytes, cudaMemcpyDeviceToDevice, st));
  if (uc_out) CUDA_TRY(cudaMemcpyAsync(uc_out, h->w.uc, bytes, cudaMemcpyDeviceToDevice, st));
  return BDDC_OK;
}

int bddc_profile_apply(bddc_handle_t h, const double* r, double* z, int32_t nrhs, int32_t reps, double* out_ms,
                       void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!r || !z || !out_ms || reps < 1) return fail(BDDC_ERR_INVALID_ARG, "bad profile arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev[10];
  for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
  for (int i = 0; i < 9; ++i) out_ms[i] = 0;
  // per-launch times need the launches in sequence: the coarse overlap (the
  // interface operator on a second stream) is off while profiling
  const int keep_overlap = h->tune_overlap;
  h->tune_overlap = 0;
  std::vector<float> t(9 * (size_t)reps, 0.0f);
  for (int rep = 0; rep < reps && rc == BDDC_OK; ++rep) {
    cudaError_t e = launch_apply(h, r, z, nrhs, st, ev);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[9]);
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&t[(size_t)i * reps + rep], ev[i], ev[i + 1]);
    if (e != cudaSuccess) rc = fail(BDDC_ERR_CUDA, cudaGetErrorString(e));
  }
  // the median of the repetitions (robust to a late launch on a busy host)
  for (int i = 0; i < 9 && rc == BDDC_OK; ++i) {
    float* b = &t[(size_t)i * reps];
    std::nth_element(b, b + reps / 2, b + reps);
    out_ms[i] = b[reps / 2];
  }
  h->tune_overlap = keep_overlap;
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

// Capture one PCG iteration (apply, beta, p update, SpMV with alpha, x/r
// update with the stop test, flag read-back) as a CUDA graph for x, nrhs,
// rtol and the form; reused while those stay the same.
static int capture_iteration(bddc_handle_t h, double* x, int nrhs, double rtol, int flexible) {
  if (h->iter_graph && h->graph_x == x && h->graph_nrhs == nrhs && h->graph_rtol == rtol &&
      h->graph_flexible == flexible)
    return BDDC_OK;
  if (h->iter_graph) {
    cudaGraphExecDestroy(h->iter_graph);
    h->iter_graph = nullptr;
  }
  if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const int R = h->nrhs_max;
  cudaStream_t cs = h->cap_stream;
  const int64_t l0 = h->launches;
  CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  cudaError_t e = launch_apply(h, h->p_r, h->p_z, nrhs, cs);
  if (e == cudaSuccess)
    e = launch_dots_fin(h, nrhs, h->p_r, h->p_z, h->p_r, h->p_zold, FIN_BETA, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_update_p(h, nrhs, cs);
  if (e == cudaSuccess) e = launch_spmv(h, h->p_p, h->p_q, nrhs, FIN_ALPHA, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_update_xr_conv(h, x, nrhs, rtol, flexible, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_flags, h->d_iscal + I_COUNT * R, kGlobalFlags * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, cs);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  h->graph_launches = h->launches - l0;
  h->launches = l0;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(BDDC_ERR_CUDA, std::string("capture of the PCG iteration: ") +
                                   cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&h->iter_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->iter_graph = nullptr;
    return fail(BDDC_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
  }
  h->graph_x = x; h->graph_nrhs = nrhs; h->graph_rtol = rtol; h->graph_flexible = flexible;
  return BDDC_OK;
}

// The whole solve as one CUDA graph: x0 = P_I b, r0, the first iteration
// (beta = 0), then a conditional WHILE node whose body is one PCG iteration
// followed by the loop-control kernel that sets its condition on the device.
// Returns OK, or BDDC_ERR_CUDA if this driver cannot build conditional
// nodes (the caller then falls back to replaying one iteration at a time).
static int capture_solve(bddc_handle_t h, const double* b, double* x, int nrhs, double rtol, int maxit,
                         int flexible) {
  if (h->solve_graph && h->solve_b == b && h->solve_x == x && h->solve_nrhs == nrhs && h->solve_rtol == rtol &&
      h->solve_maxit == maxit && h->solve_flexible == flexible)
    return BDDC_OK;
  if (h->solve_graph) {
    cudaGraphExecDestroy(h->solve_graph);
    h->solve_graph = nullptr;
  }
  if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (!h->body_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
  cudaStream_t cs = h->cap_stream, bs = h->body_stream;
  const int64_t l0 = h->launches;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(BDDC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle cond = 0;
  e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, g, 0, 0);
  // prologue and first iteration
  if (e == cudaSuccess) e = launch_interior_correction(h, b, x, nrhs, cs);
  if (e == cudaSuccess) e = launch_spmv(h, x, h->p_q, nrhs, -1, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_residual(h, b, nrhs, cs);
  if (e == cudaSuccess) e = launch_dots_fin(h, nrhs, b, b, h->p_r, h->p_r, FIN_INIT, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_apply(h, h->p_r, h->p_z, nrhs, cs);
  if (e == cudaSuccess) e = launch_dots_fin(h, nrhs, h->p_r, h->p_z, nullptr, nullptr, FIN_RHO, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_update_p(h, nrhs, cs);
  if (e == cudaSuccess) e = launch_spmv(h, h->p_p, h->p_q, nrhs, FIN_ALPHA, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_update_xr_conv(h, x, nrhs, rtol, flexible, cs);
  if (e == cudaSuccess) e = launch_loop_control(h, maxit, 1, cond, cs);
  const int64_t l1 = h->launches;
  // the loop
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps);
  cudaGraphNodeParams cp = {};
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    h->aux_sel = 1;   // the prologue's capture (on set 0) is still open
    cudaError_t eb = launch_apply(h, h->p_r, h->p_z, nrhs, bs);
    h->aux_sel = 0;
    if (eb == cudaSuccess)
      eb = launch_dots_fin(h, nrhs, h->p_r, h->p_z, h->p_r, h->p_zold, FIN_BETA, rtol, flexible, bs);
    if (eb == cudaSuccess) eb = launch_update_p(h, nrhs, bs);
    if (eb == cudaSuccess) eb = launch_spmv(h, h->p_p, h->p_q, nrhs, FIN_ALPHA, rtol, flexible, bs);
    if (eb == cudaSuccess) eb = launch_update_xr_conv(h, x, nrhs, rtol, flexible, bs);
    if (eb == cudaSuccess) eb = launch_loop_control(h, maxit, 0, cond, bs);
    cudaGraph_t body = nullptr;
    cudaError_t ee = cudaStreamEndCapture(bs, &body);
    e = eb != cudaSuccess ? eb : ee;
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  const int64_t l2 = h->launches;
  cudaGraph_t whole = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &whole);
  h->launches = l0;
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->solve_graph, whole, 0);
  if (whole) cudaGraphDestroy(whole);
  if (e != cudaSuccess) {
    h->solve_graph = nullptr;
    cudaGetLastError();
    return fail(BDDC_ERR_CUDA, std::string("whole-solve graph: ") + cudaGetErrorString(e));
  }
  h->solve_pro_launches = l1 - l0;
  h->solve_body_launches = l2 - l1;
  h->solve_b = b; h->solve_x = x; h->solve_nrhs = nrhs; h->solve_rtol = rtol; h->solve_maxit = maxit;
  h->solve_flexible = flexible;
  return BDDC_OK;
}

// per-column results of pcg_core
static int pcg_finish(bddc_handle_t h, int nrhs, int32_t* iters, double* relres, cudaStream_t st, int status) {
  const int R = h->nrhs_max;
  std::vector<int32_t> hi(I_COUNT * R + kGlobalFlags);
  std::vector<double> hd(S_COUNT * R);
  CUDA_TRY(cudaMemcpyAsync(hi.data(), h->d_iscal, hi.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hd.data(), h->d_scal, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < nrhs; ++k) {
    if (iters) iters[k] = hi[I_ITERS * R + k];
    if (relres) relres[k] = hd[S_RELRES * R + k];
    if (hi[I_STATUS * R + k] == BDDC_ERR_BREAKDOWN) status = BDDC_ERR_BREAKDOWN;
  }
  if (status == BDDC_ERR_BREAKDOWN) g_last_error = "PCG breakdown in at least one column";
  return status;
}

static int pcg_core(bddc_handle_t h, const double* b, double* x, int nrhs, double rtol, int maxit,
                    int32_t* iters, double* relres, cudaStream_t st) {
  // flexible PCG for the low-precision operators and for the inexact coarse
  // solve (a preconditioner that varies with r)
  const int flexible = h->precision != BDDC_PREC_FP64 || h->coarse_cg;
  int32_t* hf = h->h_flags;
  const int R = h->nrhs_max;
  auto read_flags = [&]() -> int {
    CUDA_TRY(cudaMemcpyAsync(hf, h->d_iscal + I_COUNT * R, kGlobalFlags * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hf[2]) return fail(BDDC_ERR_TIMEOUT, "a bounded device wait ran out");
    return BDDC_OK;
  };
  auto finish = [&](int status) { return pcg_finish(h, nrhs, iters, relres, st, status); };
  int rc;
  // iteration history: all NaN (0xff bytes) until the solve writes it
  if (h->d_hist)
    CUDA_TRY(cudaMemsetAsync(h->d_hist, 0xff, sizeof(double) * 3 * (h->hist_cap + 1) * R, st));
  int status = BDDC_OK;
  if (h->use_graph && maxit > 0 && !h->solve_graph_unsupported) {
    if ((rc = capture_solve(h, b, x, nrhs, rtol, maxit, flexible)) != BDDC_OK) {
      h->solve_graph_unsupported = true;   // fall back to one captured iteration at a time
    } else {
      CUDA_TRY(cudaGraphLaunch(h->solve_graph, st));
      if ((rc = read_flags())) return rc;
      h->launches += h->solve_pro_launches + (int64_t)std::max(hf[3] - 1, 0) * h->solve_body_launches;
      if (hf[0] > 0) status = BDDC_NOT_CONVERGED;
      return finish(status);
    }
  }
  // x0 = P_I b ; r0 = b - A x0
  CUDA_TRY(launch_interior_correction(h, b, x, nrhs, st));
  CUDA_TRY(launch_spmv(h, x, h->p_q, nrhs, -1, rtol, flexible, st));
  CUDA_TRY(launch_residual(h, b, nrhs, st));
  CUDA_TRY(launch_dots_fin(h, nrhs, b, b, h->p_r, h->p_r, FIN_INIT, rtol, flexible, st));
  rc = read_flags();
  if (rc) return rc;
  if (hf[0] > 0 && maxit > 0) {
    // first iteration launched directly, the rest replay a captured graph
    CUDA_TRY(launch_apply(h, h->p_r, h->p_z, nrhs, st));
    CUDA_TRY(launch_dots_fin(h, nrhs, h->p_r, h->p_z, nullptr, nullptr, FIN_RHO, rtol, flexible, st));
    CUDA_TRY(launch_update_p(h, nrhs, st));     // beta = 0: p = z, zold = z
    CUDA_TRY(launch_spmv(h, h->p_p, h->p_q, nrhs, FIN_ALPHA, rtol, flexible, st));
    CUDA_TRY(launch_update_xr_conv(h, x, nrhs, rtol, flexible, st));
    if ((rc = read_flags())) return rc;
    int it = 1;
    if (hf[0] > 0 && it < maxit && h->use_graph) {
      if ((rc = capture_iteration(h, x, nrhs, rtol, flexible))) return rc;
      for (; it < maxit && hf[0] > 0; ++it) {
        CUDA_TRY(cudaGraphLaunch(h->iter_graph, st));
        h->launches += h->graph_launches;
        CUDA_TRY(cudaStreamSynchronize(st));
        if (hf[2]) return fail(BDDC_ERR_TIMEOUT, "a bounded device wait ran out");
      }
    }
    for (; it < maxit && hf[0] > 0; ++it) {
      // the same iteration, launched directly
      CUDA_TRY(launch_apply(h, h->p_r, h->p_z, nrhs, st));
      CUDA_TRY(launch_dots_fin(h, nrhs, h->p_r, h->p_z, h->p_r, h->p_zold, FIN_BETA, rtol, flexible, st));
      CUDA_TRY(launch_update_p(h, nrhs, st));
      CUDA_TRY(launch_spmv(h, h->p_p, h->p_q, nrhs, FIN_ALPHA, rtol, flexible, st));
      CUDA_TRY(launch_update_xr_conv(h, x, nrhs, rtol, flexible, st));
      if ((rc = read_flags())) return rc;
    }
    if (hf[0] > 0) status = BDDC_NOT_CONVERGED;
  } else if (hf[0] > 0) {
    status = BDDC_NOT_CONVERGED;
  }
  return finish(status);
}

int bddc_pcg_solve(bddc_handle_t h, const double* b, double* x, int32_t nrhs, double rtol, int32_t maxit,
                   int32_t* iters, double* relres, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!b || !x || b == x) return fail(BDDC_ERR_INVALID_ARG, "b and x must be distinct device pointers");
  if (!(rtol > 0.0) || maxit < 0) return fail(BDDC_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 0");
  return pcg_core(h, b, x, nrhs, rtol, maxit, iters, relres, static_cast<cudaStream_t>(stream));
}

int bddc_pcg_solve_host(bddc_handle_t h, const double* b_host, double* x_host, int32_t nrhs, double rtol,
                        int32_t maxit, int32_t* iters, double* relres, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (!b_host || !x_host) return fail(BDDC_ERR_INVALID_ARG, "null host vector");
  if (!(rtol > 0.0) || maxit < 0) return fail(BDDC_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)h->n_nodes * nrhs * sizeof(double);
  CUDA_TRY(cudaMemcpyAsync(h->s_b, b_host, bytes, cudaMemcpyHostToDevice, st));
  int status = pcg_core(h, h->s_b, h->s_x, nrhs, rtol, maxit, iters, relres, st);
  if (status < 0) return status;
  CUDA_TRY(cudaMemcpyAsync(x_host, h->s_x, bytes, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return status;
}

int bddc_pcg_history(bddc_handle_t h, int32_t nrhs, int32_t n_iter, double* rnorm, double* alpha, double* beta) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  if (n_iter < 0 || n_iter > h->hist_cap)
    return fail(BDDC_ERR_INVALID_ARG, "n_iter " + std::to_string(n_iter) + " outside [0, history=" +
                                          std::to_string(h->hist_cap) + "]");
  const int R = h->nrhs_max;
  const size_t per = (size_t)(h->hist_cap + 1) * R;
  std::vector<double> hv(h->d_hist ? 3 * per : 0);
  if (h->d_hist) CUDA_TRY(cudaMemcpy(hv.data(), h->d_hist, hv.size() * sizeof(double), cudaMemcpyDeviceToHost));
  double* out[3] = {rnorm, alpha, beta};
  for (int slot = 0; slot < 3; ++slot) {
    if (!out[slot]) continue;
    for (int k = 0; k <= n_iter; ++k)
      for (int j = 0; j < nrhs; ++j)
        out[slot][(size_t)k * nrhs + j] = h->d_hist ? hv[slot * per + (size_t)k * R + j] : std::nan("");
  }
  return BDDC_OK;
}

int bddc_test_coarse_stall(bddc_handle_t h, int32_t enable, int64_t limit_cycles) {
  if (!h) return fail(BDDC_ERR_INVALID_ARG, "null handle");
  if (enable != 0 && enable != 1) return fail(BDDC_ERR_INVALID_ARG, "enable must be 0 or 1");
  if (enable && (limit_cycles < 1 || limit_cycles > kBarrierWaitCycles))
    return fail(BDDC_ERR_INVALID_ARG, "limit_cycles must be in [1, 4e9]");
  if (!h->n_c || h->coarse_dense) return fail(BDDC_ERR_INVALID_ARG, "needs the sparse coarse solve");
  ENTER_DEVICE(h->device);
  CUDA_TRY(cudaDeviceSynchronize());   // no coarse launch in flight while the arguments change
  h->cbar_extra = enable ? 1u : 0u;
  h->cbar_cycles = enable ? (long long)limit_cycles : kBarrierWaitCycles;
  drop_graphs(h);
  return BDDC_OK;
}

int bddc_clear_device_error(bddc_handle_t h) {
  if (!h) return fail(BDDC_ERR_INVALID_ARG, "null handle");
  ENTER_DEVICE(h->device);
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int32_t)));
  h->info.device_error = 0;
  return BDDC_OK;
}

int bddc_get_tuning(bddc_handle_t h, bddc_tuning_t* out) {
  if (!h || !out) return fail(BDDC_ERR_INVALID_ARG, "null handle or output");
  *out = bddc_tuning_t{h->tune_stage_kb[0], h->tune_stage_kb[1], h->tune_coarse_rb_min,
                       64 << h->tune_tile_class[0], 64 << h->tune_tile_class[1], h->tune_overlap,
                       h->tune_sym_stages[0], h->tune_sym_stages[1], h->is.block_min_height,
                       h->cs.use_level ? 1 : 0};
  return BDDC_OK;
}

int bddc_set_tuning(bddc_handle_t h, const bddc_tuning_t* in) {
  if (!h || !in) return fail(BDDC_ERR_INVALID_ARG, "null handle or input");
  if (in->gemv_stage_kb_interior < 1 || in->gemv_stage_kb_interior > 64 || in->gemv_stage_kb_interface < 1 ||
      in->gemv_stage_kb_interface > 64)
    return fail(BDDC_ERR_INVALID_ARG, "GEMV stage size must be 1..64 KB");
  if (in->coarse_rowblock_min_nrhs < 2 || in->coarse_rowblock_min_nrhs > 65)
    return fail(BDDC_ERR_INVALID_ARG, "coarse row-blocking threshold must be 2..65");
  auto tile_class = [](int rows) { return rows == 64 ? 0 : rows == 128 ? 1 : rows == 256 ? 2 : -1; };
  if (tile_class(in->gemv_rows_interior) < 0 || tile_class(in->gemv_rows_interface) < 0)
    return fail(BDDC_ERR_INVALID_ARG, "GEMV row tile must be 64, 128 or 256");
  if (in->coarse_overlap != 0 && in->coarse_overlap != 1)
    return fail(BDDC_ERR_INVALID_ARG, "coarse_overlap must be 0 or 1");
  if (in->sym_stages_interior < 3 || in->sym_stages_interior > 4 || in->sym_stages_interface < 3 ||
      in->sym_stages_interface > 4)
    return fail(BDDC_ERR_INVALID_ARG, "symmetric GEMV stages must be 3 or 4");
  if (in->interior_block_height < 0 || in->interior_block_height > 64)
    return fail(BDDC_ERR_INVALID_ARG, "interior_block_height must be 0..64");
  if (in->coarse_level_launches != 0 && in->coarse_level_launches != 1)
    return fail(BDDC_ERR_INVALID_ARG, "coarse_level_launches must be 0 or 1");
  h->tune_tile_class[0] = tile_class(in->gemv_rows_interior);
  h->tune_tile_class[1] = tile_class(in->gemv_rows_interface);
  h->tune_overlap = in->coarse_overlap;
  h->tune_stage_kb[0] = in->gemv_stage_kb_interior;
  h->tune_stage_kb[1] = in->gemv_stage_kb_interface;
  h->tune_sym_stages[0] = in->sym_stages_interior;
  h->tune_sym_stages[1] = in->sym_stages_interface;
  h->tune_coarse_rb_min = in->coarse_rowblock_min_nrhs;
  h->cs.use_level = in->coarse_level_launches == 1 && !h->cs.lv.empty();
  if (h->is.block_form) {
    // the interior sweeps' bytes per solve follow the split
    const int64_t before = sweep_read_1col(h->is);
    h->is.block_min_height = std::min(in->interior_block_height, h->is.levels);
    const int64_t after = sweep_read_1col(h->is);
    h->info.interior_op_bytes = after;
    h->info.apply_bytes_1rhs += 2 * (after - before);
  }
  drop_graphs(h);   // captured graphs hold the old launch parameters
  return BDDC_OK;
}

int bddc_autotune(bddc_handle_t h, int32_t nrhs, bddc_tuning_t* out, void* stream) {
  int rc = check_handle(h, nrhs);
  if (rc) return rc;
  ENTER_DEVICE(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  // time `reps` launches of f after one warm-up launch; the median of 3 rounds
  auto timed = [&](auto&& f) -> float {
    if (f() != cudaSuccess) return -1.0f;
    float best[3];
    for (int round = 0; round < 3; ++round) {
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r)
        if (f() != cudaSuccess) return -1.0f;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
      cudaEventElapsedTime(&best[round], e0, e1);
    }
    std::sort(best, best + 3);
    return best[1];
  };
  bddc_tuning_t t{h->tune_stage_kb[0], h->tune_stage_kb[1], h->tune_coarse_rb_min, 64 << h->tune_tile_class[0],
                  64 << h->tune_tile_class[1], h->tune_overlap, h->tune_sym_stages[0], h->tune_sym_stages[1],
                  h->is.block_min_height, h->cs.use_level ? 1 : 0};
  cudaError_t ce = cudaSuccess;
  if ((ce = cudaMemsetAsync(h->w.rI, 0, sizeof(double) * std::max<int64_t>(h->nI_tot, 1) * nrhs, st)) ||
      (ce = cudaMemsetAsync(h->w.yG, 0, sizeof(double) * std::max<int64_t>(h->nG_tot, 1) * nrhs, st))) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(BDDC_ERR_CUDA, cudaGetErrorString(ce));
  }
  if (h->use_tma && !h->use_tc) {
    // every (row tile, stage size) pair of each operator family; for the
    // symmetric GEMV (one work item per operator) every (stages, stage size)
    // pair instead
    const int cand[4] = {6, 12, 24, 48};
    const int sym_cand[7][2] = {{4, 10}, {4, 12}, {4, 16}, {4, 20}, {3, 16}, {3, 20}, {3, 24}};
    for (int fam = 0; fam < 2; ++fam) {
      const bool interior = fam == 0;
      if ((interior ? h->nI_tot : h->nG_tot) == 0) continue;
      if (interior && h->sparse_local) continue;   // the interior solves are sweeps, not a GEMV
      float best = -1.0f;
      int best_kb = h->tune_stage_kb[fam], best_tc = h->tune_tile_class[fam], best_ns = h->tune_sym_stages[fam];
      auto try_one = [&](int kb, int tc, int ns) {
        h->tune_stage_kb[fam] = kb;
        h->tune_tile_class[fam] = tc;
        h->tune_sym_stages[fam] = ns;
        const float ms = timed([&] {
          return launch_local_op(h, interior, interior ? h->w.rI : h->w.yG, interior ? h->w.tI : h->w.zG, nrhs, st);
        });
        if (ms >= 0.0f && (best < 0.0f || ms < best)) {
          best = ms;
          best_kb = kb;
          best_tc = tc;
          best_ns = ns;
        }
      };
      if (h->use_sym) {
        for (const auto& c : sym_cand) try_one(c[1], best_tc, c[0]);
      } else {
        for (int tc = 0; tc < 3; ++tc)
          for (int c : cand) try_one(c, tc, best_ns);
      }
      h->tune_stage_kb[fam] = best_kb;
      h->tune_tile_class[fam] = best_tc;
      h->tune_sym_stages[fam] = best_ns;
      (interior ? t.gemv_stage_kb_interior : t.gemv_stage_kb_interface) = best_kb;
      (interior ? t.gemv_rows_interior : t.gemv_rows_interface) = 64 << best_tc;
      (interior ? t.sym_stages_interior : t.sym_stages_interface) = best_ns;
    }
  }
  if (h->is.block_form && nrhs == 1 && h->nI_tot) {
    // every split height of the interior sweeps (one interior solve each)
    const int keep = h->is.block_min_height;
    float best = -1.0f;
    int best_k = keep;
    for (int k = 0; k <= h->is.levels; ++k) {
      h->is.block_min_height = k;
      const float ms = timed([&] { return launch_local_op(h, true, h->w.rI, h->w.tI, 1, st); });
      if (ms >= 0.0f && (best < 0.0f || ms < best)) {
        best = ms;
        best_k = k;
      }
    }
    h->is.block_min_height = keep;
    t.interior_block_height = best_k;
  }
  if (h->n_c && !h->coarse_dense && !h->coarse_cg && nrhs == 1 && !h->cs.lv.empty()) {
    // one cooperative launch against one launch per level
    CUDA_TRY(cudaMemsetAsync(h->w.rc, 0, sizeof(double) * h->n_c, st));
    const bool keep = h->cs.use_level;
    h->cs.use_level = false;
    const float coop = timed([&] { return launch_coarse_solve(h, h->w, h->w.rc, h->w.uc, 1, st); });
    h->cs.use_level = true;
    const float lev = timed([&] { return launch_coarse_solve(h, h->w, h->w.rc, h->w.uc, 1, st); });
    h->cs.use_level = keep;
    if (coop >= 0.0f && lev >= 0.0f) t.coarse_level_launches = lev < coop ? 1 : 0;
  }
  if (h->n_c && !h->coarse_dense && !h->coarse_cg && nrhs >= 2) {
    CUDA_TRY(cudaMemsetAsync(h->w.rc, 0, sizeof(double) * h->n_c * nrhs, st));
    const int keep = h->tune_coarse_rb_min;
    h->tune_coarse_rb_min = nrhs;   // blocked
    const float blocked = timed([&] { return launch_coarse_solve(h, h->w, h->w.rc, h->w.uc, nrhs, st); });
    h->tune_coarse_rb_min = 65;     // one row per unit
    const float single = timed([&] { return launch_coarse_solve(h, h->w, h->w.rc, h->w.uc, nrhs, st); });
    h->tune_coarse_rb_min = keep;
    if (blocked >= 0.0f && single >= 0.0f)
      t.coarse_rowblock_min_nrhs = blocked < single ? std::min(keep, (int)nrhs) : std::max(keep, (int)nrhs + 1);
  }
  // whole applies with and without the coarse overlap (after the choices above)
  if (h->aux_stream[0] && h->n_c && !h->coarse_dense && h->nG_tot) {
    h->tune_stage_kb[0] = t.gemv_stage_kb_interior;
    h->tune_stage_kb[1] = t.gemv_stage_kb_interface;
    h->tune_coarse_rb_min = t.coarse_rowblock_min_nrhs;
    h->cs.use_level = t.coarse_level_launches == 1 && !h->cs.lv.empty();
    h->is.block_min_height = std::min(t.interior_block_height, h->is.levels);
    double* rz = nullptr;
    const size_t nv = (size_t)h->n_nodes * nrhs;
    if (cudaMalloc(&rz, 2 * nv * sizeof(double)) == cudaSuccess) {
      cudaMemsetAsync(rz, 0, 2 * nv * sizeof(double), st);
      const int keep = h->tune_overlap;
      h->tune_overlap = 0;
      const float plain = timed([&] { return launch_apply(h, rz, rz + nv, nrhs, st); });
      h->tune_overlap = 1;
      const float over = timed([&] { return launch_apply(h, rz, rz + nv, nrhs, st); });
      h->tune_overlap = keep;
      if (plain >= 0.0f && over >= 0.0f) t.coarse_overlap = over < plain ? 1 : 0;
      cudaStreamSynchronize(st);
      cudaFree(rz);
    } else {
      cudaGetLastError();
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaGetLastError());
  if ((rc = bddc_set_tuning(h, &t)) != BDDC_OK) return rc;
  if (out) *out = t;
  return BDDC_OK;
}

}  // extern "C"
