// Host-side setup of the BDDC preconditioner, all in float64.
//
// Topology (Sec. 2 of arXiv 2410.14786): subdomain node sets from the
// element partition, multiplicities kappa (weights 1/kappa), the split of
// each subdomain's free nodes into interior (kappa = 1) and interface
// (kappa >= 2) nodes, and the globs: interface nodes with the same set of
// sharing subdomains, split into mesh-connected pieces. A single-node glob
// is a corner (point constraint); larger ones are edges or faces (averages
// with weight 1/|G|).
//
// Numerics per subdomain, with A_i ordered [interior I; interface G]:
//   A_II^-1                                   explicit, for the interior solves
//   S   = A_GG - A_GI A_II^-1 A_IG            local Schur complement
//   Ahat = S + rho C^T C                      SPD, same saddle-point solutions
//   G   = Ahat^-1 C^T,  Sc = C G
//   Phi_G = G Sc^-1                            interface rows of Phi_i (Eq. saddlepoint)
//   A_ci  = Sc^-1 - rho I                      = Phi_i^T A_i Phi_i = -Lambda_i
//   K_GG  = Ahat^-1 - Phi_G G^T                (1,1) block of [S C^T; C 0]^-1
// With the sparse local solver A_II^-1 is never formed: A_i is assembled in
// CSR and factorised by the supernodal Cholesky of coarse_sparse.cpp in
// nested-dissection order of the subdomain's elements, the interface dofs
// eliminated last; their front, assembled but not factorised, is S (the
// same matrix, without the dense n_I x n_I inverse), and the factor of A_II
// is kept for the interior sweeps on the device.
// The interior rows of Phi_i and z_i follow from the first block row,
// x_I = A_II^-1 (y_I - A_IG x_G), and are never stored (see the apply).
// Coarse: A_c = sum_i R_ci^T A_ci R_ci, factorised by the sparse Cholesky of
// coarse_sparse.cpp (default), inverted explicitly (dense option), or kept
// in CSR for the inexact solve by plain CG.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>

#include "dense.hpp"
#include "internal.hpp"

namespace bddc {

namespace {

// Q1 element stiffness for unit sigma on an element of side h, as a
// function of the Hamming distance between the local nodes' corner bits:
// 2D: (1/6)[4, -1, -2]; 3D: h * [1/3, 0, -1/12, -1/12].
void q1_stiffness_by_distance(int dim, double h, double out[4]) {
  if (dim == 2) {
    out[0] = 4.0 / 6.0; out[1] = -1.0 / 6.0; out[2] = -2.0 / 6.0; out[3] = 0.0;
  } else {
    out[0] = h / 3.0; out[1] = 0.0; out[2] = -h / 12.0; out[3] = -h / 12.0;
  }
}

struct DSU {
  std::vector<int32_t> p;
  explicit DSU(size_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int32_t find(int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  void unite(int32_t a, int32_t b) {
    a = find(a); b = find(b);
    if (a != b) { if (a < b) p[b] = a; else p[a] = b; }
  }
};

}  // namespace

int validate_problem(const bddc_problem_t* P, const bddc_options_t* O, std::string& err) {
  if (!P || !O) { err = "null argument"; return BDDC_ERR_INVALID_ARG; }
  if (P->dim != 2 && P->dim != 3) { err = "dim must be 2 or 3"; return BDDC_ERR_INVALID_ARG; }
  if (P->ne < 1 || P->ne > (P->dim == 2 ? 20000 : 1000)) { err = "ne out of range"; return BDDC_ERR_INVALID_ARG; }
  if (P->n_sub < 1) { err = "n_sub must be >= 1"; return BDDC_ERR_INVALID_ARG; }
  if (!P->elem_sigma || !P->elem_subdomain) { err = "null problem arrays"; return BDDC_ERR_INVALID_ARG; }
  if (O->precision < BDDC_PREC_FP64 || O->precision > BDDC_PREC_TF32) { err = "unknown precision"; return BDDC_ERR_INVALID_ARG; }
  if (O->tensor_cores < BDDC_TC_AUTO || O->tensor_cores > BDDC_TC_OFF) { err = "unknown tensor_cores mode"; return BDDC_ERR_INVALID_ARG; }
  if (O->tensor_cores == BDDC_TC_OFF && O->precision == BDDC_PREC_TF32) { err = "TF32 needs the tensor cores"; return BDDC_ERR_INVALID_ARG; }
  if (O->tensor_cores == BDDC_TC_ON && (O->precision == BDDC_PREC_FP64 || O->precision == BDDC_PREC_FP32)) { err = "tensor cores run the BF16 and TF32 forms only"; return BDDC_ERR_INVALID_ARG; }
  if (O->nrhs_max < 1 || O->nrhs_max > 64) { err = "nrhs_max must be in [1, 64]"; return BDDC_ERR_INVALID_ARG; }
  if (O->constraints & ~7u) { err = "unknown constraint bits"; return BDDC_ERR_INVALID_ARG; }
  if (O->coarse < BDDC_COARSE_AUTO || O->coarse > BDDC_COARSE_CG) { err = "unknown coarse mode"; return BDDC_ERR_INVALID_ARG; }
  if (O->coarse_cg_maxit < 0) { err = "coarse_cg_maxit must be >= 0"; return BDDC_ERR_INVALID_ARG; }
  if (!(O->coarse_cg_rtol >= 0.0 && O->coarse_cg_rtol < 1.0)) { err = "coarse_cg_rtol must be in [0, 1)"; return BDDC_ERR_INVALID_ARG; }
  if (O->coarse_blocks < 0) { err = "coarse_blocks must be >= 0"; return BDDC_ERR_INVALID_ARG; }
  if (O->full_operators != 0 && O->full_operators != 1) { err = "full_operators must be 0 or 1"; return BDDC_ERR_INVALID_ARG; }
  if (O->local_solver != BDDC_LOCAL_DENSE && O->local_solver != BDDC_LOCAL_SPARSE) { err = "unknown local_solver"; return BDDC_ERR_INVALID_ARG; }
  if (O->local_leaf < 0 || O->local_leaf > 4096) { err = "local_leaf must be in [0, 4096]"; return BDDC_ERR_INVALID_ARG; }
  if (O->history < 0 || O->history > 100000) { err = "history must be in [0, 100000]"; return BDDC_ERR_INVALID_ARG; }
  const int64_t ne = P->ne;
  const int64_t n_el = P->dim == 2 ? ne * ne : ne * ne * ne;
  for (int64_t e = 0; e < n_el; ++e) {
    const double s = P->elem_sigma[e];
    if (!(s > 0.0) || !std::isfinite(s)) {
      err = "elem_sigma[" + std::to_string(e) + "] is not finite and positive";
      return BDDC_ERR_INVALID_ARG;
    }
    if (P->elem_subdomain[e] < 0 || P->elem_subdomain[e] >= P->n_sub) {
      err = "elem_subdomain[" + std::to_string(e) + "] out of range";
      return BDDC_ERR_INVALID_ARG;
    }
  }
  return BDDC_OK;
}

int host_setup(const bddc_problem_t* P, const bddc_options_t* O, HostSetup& hs, std::string& err,
               bool factor_coarse, bool numerics) {
  const int dim = P->dim, ne = P->ne;
  hs.dim = dim; hs.ne = ne; hs.n1 = ne + 1;
  const int64_t n1 = ne + 1;
  hs.n_nodes = dim == 2 ? n1 * n1 : n1 * n1 * n1;
  hs.n_elems = dim == 2 ? (int64_t)ne * ne : (int64_t)ne * ne * ne;
  hs.h = 1.0 / ne;
  hs.n_sub = P->n_sub;
  const int nloc = 1 << dim;
  const int maxs = nloc;     // a node touches at most 2^dim elements
  int threads = O->n_threads > 0 ? O->n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  uint32_t mask = O->constraints ? O->constraints : (BDDC_CORNERS | BDDC_EDGES | BDDC_FACES);

  auto node_id = [&](int64_t ix, int64_t iy, int64_t iz) { return ix + n1 * (iy + n1 * iz); };
  auto elem_node = [&](int64_t e, int a) {
    int64_t ex = e % ne, ey = (e / ne) % ne, ez = dim == 3 ? e / ((int64_t)ne * ne) : 0;
    return node_id(ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1));
  };
  auto is_dir = [&](int64_t n) {
    int64_t ix = n % n1, iy = (n / n1) % n1, iz = dim == 3 ? n / (n1 * n1) : 1;
    bool d = ix == 0 || ix == ne || iy == 0 || iy == ne;
    if (dim == 3) d = d || iz == 0 || iz == ne;
    return d;
  };

  // ---- elements per subdomain -------------------------------------------
  std::vector<int64_t> sptr(hs.n_sub + 1, 0);
  for (int64_t e = 0; e < hs.n_elems; ++e) sptr[P->elem_subdomain[e] + 1]++;
  for (int s = 0; s < hs.n_sub; ++s) {
    if (sptr[s + 1] == 0) { err = "subdomain " + std::to_string(s) + " has no elements"; return BDDC_ERR_INVALID_ARG; }
    sptr[s + 1] += sptr[s];
  }
  std::vector<int32_t> selem(hs.n_elems);
  {
    std::vector<int64_t> fill(sptr.begin(), sptr.end() - 1);
    for (int64_t e = 0; e < hs.n_elems; ++e) selem[fill[P->elem_subdomain[e]]++] = (int32_t)e;
  }

  // ---- sharing sets and multiplicity --------------------------------------
  std::vector<int32_t> nsubs((size_t)hs.n_nodes * maxs, -1);
  hs.kappa.assign(hs.n_nodes, 0);
  for (int64_t e = 0; e < hs.n_elems; ++e) {
    int32_t s = P->elem_subdomain[e];
    for (int a = 0; a < nloc; ++a) {
      int64_t n = elem_node(e, a);
      int32_t* lst = &nsubs[(size_t)n * maxs];
      int k = 0;
      while (k < maxs && lst[k] >= 0 && lst[k] != s) ++k;
      if (k < maxs && lst[k] < 0) lst[k] = s;
    }
  }
  for (int64_t n = 0; n < hs.n_nodes; ++n) {
    int32_t* lst = &nsubs[(size_t)n * maxs];
    int k = 0;
    while (k < maxs && lst[k] >= 0) ++k;
    std::sort(lst, lst + k);
    if (is_dir(n)) { hs.dir_nodes.push_back((int32_t)n); hs.kappa[n] = 0; }
    else hs.kappa[n] = (uint8_t)k;
  }

  // ---- subdomain interior / interface node lists ------------------------
  hs.sub_I.assign(hs.n_sub, {});
  hs.sub_G.assign(hs.n_sub, {});
  parallel_for(hs.n_sub, threads, [&](int64_t s) {
    std::vector<int32_t> nodes;
    nodes.reserve((sptr[s + 1] - sptr[s]) * 2);
    for (int64_t q = sptr[s]; q < sptr[s + 1]; ++q)
      for (int a = 0; a < nloc; ++a) nodes.push_back((int32_t)elem_node(selem[q], a));
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    for (int32_t n : nodes) {
      if (hs.kappa[n] == 0) continue;
      (hs.kappa[n] == 1 ? hs.sub_I[s] : hs.sub_G[s]).push_back(n);
    }
  });

  // ---- globs ----------------------------------------------------------------
  {
    DSU dsu((size_t)hs.n_nodes);
    const int64_t strides[3] = {1, n1, n1 * n1};
    auto same_set = [&](int64_t a, int64_t b) {
      return std::memcmp(&nsubs[(size_t)a * maxs], &nsubs[(size_t)b * maxs], sizeof(int32_t) * maxs) == 0;
    };
    for (int64_t n = 0; n < hs.n_nodes; ++n) {
      if (hs.kappa[n] < 2) continue;
      int64_t c[3] = {n % n1, (n / n1) % n1, dim == 3 ? n / (n1 * n1) : 0};
      for (int d = 0; d < dim; ++d) {
        if (c[d] >= ne) continue;
        int64_t m = n + strides[d];
        if (hs.kappa[m] >= 2 && same_set(n, m)) dsu.unite((int32_t)n, (int32_t)m);
      }
    }
    // roots are the smallest member, so scanning nodes in order lists globs
    // by their smallest node id
    std::vector<int32_t> gid(hs.n_nodes, -1);
    std::vector<std::vector<int32_t>> members;
    for (int64_t n = 0; n < hs.n_nodes; ++n) {
      if (hs.kappa[n] < 2) continue;
      int32_t r = dsu.find((int32_t)n);
      if (gid[r] < 0) { gid[r] = (int32_t)members.size(); members.emplace_back(); }
      members[gid[r]].push_back((int32_t)n);
    }
    for (auto& m : members) {
      int32_t n0 = m[0];
      int k = 0;
      while (k < maxs && nsubs[(size_t)n0 * maxs + k] >= 0) ++k;
      int kind = m.size() == 1 ? BDDC_CORNERS : (dim == 3 && k == 2 ? BDDC_FACES : BDDC_EDGES);
      if (!(kind & mask)) continue;
      hs.glob_nodes.push_back(m);
      hs.glob_subs.emplace_back(&nsubs[(size_t)n0 * maxs], &nsubs[(size_t)n0 * maxs] + k);
      hs.glob_kind.push_back(kind);
    }
    hs.n_c = (int64_t)hs.glob_nodes.size();
    hs.sub_globs.assign(hs.n_sub, {});
    for (int64_t g = 0; g < hs.n_c; ++g)
      for (int32_t s : hs.glob_subs[g]) hs.sub_globs[s].push_back((int32_t)g);
  }

  if (!numerics) return BDDC_OK;

  // ---- per-subdomain numerics -----------------------------------------------
  double kd[4];
  q1_stiffness_by_distance(dim, hs.h, kd);
  const bool sparse = O->local_solver == BDDC_LOCAL_SPARSE;
  const int leaf = O->local_leaf > 0 ? O->local_leaf : kLocalLeaf;
  hs.sparse_local = sparse;
  hs.ifac.assign(sparse ? hs.n_sub : 0, {});
  hs.AIIinv.assign(hs.n_sub, {});
  hs.Kgg.assign(hs.n_sub, {});
  hs.Phi.assign(hs.n_sub, {});
  hs.Aci.assign(hs.n_sub, {});
  hs.agi_ptr.assign(hs.n_sub, {}); hs.agi_col.assign(hs.n_sub, {}); hs.agi_val.assign(hs.n_sub, {});
  hs.aig_ptr.assign(hs.n_sub, {}); hs.aig_col.assign(hs.n_sub, {}); hs.aig_val.assign(hs.n_sub, {});
  std::atomic<int> bad_sub{-1};
  // subdomains largest first, so the longest jobs start early
  std::vector<int32_t> order(hs.n_sub);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    size_t na = hs.sub_I[a].size() + hs.sub_G[a].size(), nb = hs.sub_I[b].size() + hs.sub_G[b].size();
    return na != nb ? na > nb : a < b;
  });
  parallel_for(hs.n_sub, threads, [&](int64_t t) {
    const int s = order[t];
    const auto& I = hs.sub_I[s];
    const auto& G = hs.sub_G[s];
    const int nI = (int)I.size(), nG = (int)G.size(), n = nI + nG;
    const auto& gl = hs.sub_globs[s];
    const int nc = (int)gl.size();
    // local index of each node: interior first, then interface
    auto local = [&](int32_t node) -> int {
      auto it = std::lower_bound(I.begin(), I.end(), node);
      if (it != I.end() && *it == node) return (int)(it - I.begin());
      auto jt = std::lower_bound(G.begin(), G.end(), node);
      if (jt != G.end() && *jt == node) return nI + (int)(jt - G.begin());
      return -1;
    };
    std::vector<double> S;   // Schur complement A_GG - A_GI A_II^-1 A_IG (nG x nG)
    if (sparse) {
      // local matrix in CSR (both triangles, exact zeros dropped), from the
      // subdomain's elements; rows and columns in local order [I; G]
      const int cap = dim == 2 ? 9 : 27;
      std::vector<int32_t> rc((size_t)n * cap), cnt(n, 0);
      std::vector<double> rv((size_t)n * cap, 0.0);
      std::vector<std::vector<int32_t>> groups(nI);
      const int64_t nel = sptr[s + 1] - sptr[s];
      std::vector<double> gxyz(3 * (size_t)nel);
      for (int64_t q = sptr[s]; q < sptr[s + 1]; ++q) {
        const int64_t e = selem[q], lq = q - sptr[s];
        gxyz[3 * lq] = (double)(e % ne) + 0.5;
        gxyz[3 * lq + 1] = (double)((e / ne) % ne) + 0.5;
        gxyz[3 * lq + 2] = dim == 3 ? (double)(e / ((int64_t)ne * ne)) + 0.5 : 0.0;
        int li[8];
        for (int a2 = 0; a2 < nloc; ++a2) {
          const int64_t nd = elem_node(e, a2);
          li[a2] = hs.kappa[nd] ? local((int32_t)nd) : -1;
          if (li[a2] >= 0 && li[a2] < nI) groups[li[a2]].push_back((int32_t)lq);
        }
        const double sg = P->elem_sigma[e];
        for (int a2 = 0; a2 < nloc; ++a2) {
          if (li[a2] < 0) continue;
          int32_t* cr = &rc[(size_t)li[a2] * cap];
          double* vr = &rv[(size_t)li[a2] * cap];
          for (int b2 = 0; b2 < nloc; ++b2) {
            if (li[b2] < 0) continue;
            int k = 0;
            while (k < cnt[li[a2]] && cr[k] != li[b2]) ++k;
            if (k == cnt[li[a2]]) { cr[k] = li[b2]; vr[k] = 0.0; cnt[li[a2]]++; }
            vr[k] += sg * kd[__builtin_popcount(a2 ^ b2)];
          }
        }
      }
      std::vector<int64_t> rp(n + 1, 0);
      std::vector<int32_t> ci;
      std::vector<double> cv;
      std::vector<std::pair<int32_t, double>> row;
      for (int r = 0; r < n; ++r) {
        row.clear();
        for (int k = 0; k < cnt[r]; ++k)
          if (rv[(size_t)r * cap + k] != 0.0) row.emplace_back(rc[(size_t)r * cap + k], rv[(size_t)r * cap + k]);
        std::sort(row.begin(), row.end());
        for (auto& x : row) { ci.push_back(x.first); cv.push_back(x.second); }
        rp[r + 1] = (int64_t)ci.size();
      }
      std::vector<int32_t>().swap(rc);
      std::vector<double>().swap(rv);
      // sparse couplings between interior and interface
      auto& gp = hs.agi_ptr[s]; auto& gc = hs.agi_col[s]; auto& gv = hs.agi_val[s];
      gp.assign(nG + 1, 0);
      for (int r = 0; r < nG; ++r) {
        for (int64_t j = rp[nI + r]; j < rp[nI + r + 1]; ++j)
          if (ci[j] < nI) { gc.push_back(ci[j]); gv.push_back(cv[j]); }
        gp[r + 1] = (int32_t)gc.size();
      }
      auto& ip = hs.aig_ptr[s]; auto& ic = hs.aig_col[s]; auto& iv = hs.aig_val[s];
      ip.assign(nI + 1, 0);
      for (int r = 0; r < nI; ++r) {
        for (int64_t j = rp[r]; j < rp[r + 1]; ++j)
          if (ci[j] >= nI) { ic.push_back(ci[j] - nI); iv.push_back(cv[j]); }
        ip[r + 1] = (int32_t)ic.size();
      }
      // A_II factorised in nested-dissection order of the elements, the
      // interface eliminated last: its front is S
      std::string ferr;
      if (sparse_factor(n, rp, ci, cv, groups, gxyz, nG, leaf, hs.ifac[s], &S, ferr) != BDDC_OK) {
        bad_sub = s;
        return;
      }
      if (nG == 0) return;
    } else {
      std::vector<double> A((size_t)n * n, 0.0);
      for (int64_t q = sptr[s]; q < sptr[s + 1]; ++q) {
        int64_t e = selem[q];
        int li[8];
        for (int a = 0; a < nloc; ++a) {
          int64_t nd = elem_node(e, a);
          li[a] = hs.kappa[nd] ? local((int32_t)nd) : -1;
        }
        const double sg = P->elem_sigma[e];
        for (int a = 0; a < nloc; ++a) {
          if (li[a] < 0) continue;
          for (int b = 0; b < nloc; ++b) {
            if (li[b] < 0) continue;
            A[(size_t)li[a] * n + li[b]] += sg * kd[__builtin_popcount(a ^ b)];
          }
        }
      }
      // sparse couplings between interior and interface
      auto& gp = hs.agi_ptr[s]; auto& gc = hs.agi_col[s]; auto& gv = hs.agi_val[s];
      gp.assign(nG + 1, 0);
      for (int r = 0; r < nG; ++r) {
        for (int c = 0; c < nI; ++c) {
          double v = A[(size_t)(nI + r) * n + c];
          if (v != 0.0) { gc.push_back(c); gv.push_back(v); }
        }
        gp[r + 1] = (int32_t)gc.size();
      }
      auto& ip = hs.aig_ptr[s]; auto& ic = hs.aig_col[s]; auto& iv = hs.aig_val[s];
      ip.assign(nI + 1, 0);
      for (int r = 0; r < nI; ++r) {
        for (int c = 0; c < nG; ++c) {
          double v = A[(size_t)r * n + nI + c];
          if (v != 0.0) { ic.push_back(c); iv.push_back(v); }
        }
        ip[r + 1] = (int32_t)ic.size();
      }
      // interior block: Cholesky, L^-1, A_II^-1
      std::vector<double> L((size_t)nI * nI), X((size_t)nI * nI);
      for (int r = 0; r < nI; ++r) std::memcpy(&L[(size_t)r * nI], &A[(size_t)r * n], sizeof(double) * nI);
      if (nI > 0) {
        if (dense::potrf(nI, L.data(), nI) >= 0) { bad_sub = s; return; }
        dense::trtri_lower(nI, L.data(), nI, X.data(), nI);
        hs.AIIinv[s].assign((size_t)nI * nI, 0.0);
        dense::lower_gram(nI, X.data(), nI, hs.AIIinv[s].data(), nI);
      }
      if (nG == 0) return;
      // Schur complement S = A_GG - Y^T Y with Y = L^-1 A_IG
      S.assign((size_t)nG * nG, 0.0);
      for (int r = 0; r < nG; ++r)
        std::memcpy(&S[(size_t)r * nG], &A[(size_t)(nI + r) * n + nI], sizeof(double) * nG);
      if (nI > 0) {
        std::vector<double> Y((size_t)nI * nG, 0.0);
        dense::gemm_nn(nI, nG, nI, 1.0, X.data(), nI, &A[nI], n, Y.data(), nG);
        dense::gemm(dense::GemmArgs{nG, nG, nI, -1.0, Y.data(), nG, true, Y.data(), nG, false, S.data(), nG});
      }
    }
    // constraints on the interface (rows: globs of this subdomain)
    std::vector<double> C((size_t)nc * nG, 0.0);
    for (int r = 0; r < nc; ++r) {
      const auto& mem = hs.glob_nodes[gl[r]];
      const double w = 1.0 / (double)mem.size();
      for (int32_t nd : mem) {
        auto jt = std::lower_bound(G.begin(), G.end(), nd);
        C[(size_t)r * nG + (jt - G.begin())] = w;
      }
    }
    double tr = 0;
    for (int r = 0; r < nG; ++r) tr += S[(size_t)r * nG + r];
    const double rho = nc > 0 ? tr / nc : 0.0;
    std::vector<double> Ah = S;
    if (nc > 0) dense::gemm(dense::GemmArgs{nG, nG, nc, rho, C.data(), nG, true, C.data(), nG, false, Ah.data(), nG});
    // symmetrise against rounding in the products
    for (int r = 0; r < nG; ++r)
      for (int c = r + 1; c < nG; ++c) {
        double v = 0.5 * (Ah[(size_t)r * nG + c] + Ah[(size_t)c * nG + r]);
        Ah[(size_t)r * nG + c] = Ah[(size_t)c * nG + r] = v;
      }
    if (dense::spd_inverse(nG, Ah.data(), nG) >= 0) { bad_sub = s; return; }
    hs.Kgg[s] = Ah;                                  // Ahat^-1 (corrected below)
    if (nc == 0) return;
    std::vector<double> Gm((size_t)nG * nc, 0.0), Sc((size_t)nc * nc, 0.0);
    dense::gemm(dense::GemmArgs{nG, nc, nG, 1.0, Ah.data(), nG, false, C.data(), nG, true, Gm.data(), nc});
    dense::gemm_nn(nc, nc, nG, 1.0, C.data(), nG, Gm.data(), nc, Sc.data(), nc);
    for (int r = 0; r < nc; ++r)
      for (int c = r + 1; c < nc; ++c) {
        double v = 0.5 * (Sc[(size_t)r * nc + c] + Sc[(size_t)c * nc + r]);
        Sc[(size_t)r * nc + c] = Sc[(size_t)c * nc + r] = v;
      }
    if (dense::spd_inverse(nc, Sc.data(), nc) >= 0) { bad_sub = s; return; }
    hs.Phi[s].assign((size_t)nG * nc, 0.0);
    dense::gemm_nn(nG, nc, nc, 1.0, Gm.data(), nc, Sc.data(), nc, hs.Phi[s].data(), nc);
    hs.Aci[s] = Sc;
    for (int r = 0; r < nc; ++r) hs.Aci[s][(size_t)r * nc + r] -= rho;
    dense::gemm(dense::GemmArgs{nG, nG, nc, -1.0, hs.Phi[s].data(), nc, false, Gm.data(), nc, true,
                                hs.Kgg[s].data(), nG});
  });
  if (bad_sub >= 0) {
    hs.error_subdomain = bad_sub;
    err = "non-positive pivot in the local factorisations of subdomain " + std::to_string(bad_sub.load()) +
          " (a floating subdomain without constraints?)";
    return BDDC_ERR_SINGULAR;
  }

  // ---- coarse matrix (sparse) and its factorisation -------------------------------
  const int64_t nC = hs.n_c;
  if (nC > 0) {
    // CSR of A_c = sum_i R_ci^T A_ci R_ci: rows gathered from the subdomains
    // holding each coarse dof, duplicates summed
    std::vector<std::vector<int32_t>> dof_subs(nC);
    for (int s = 0; s < hs.n_sub; ++s)
      for (int r = 0; r < (int)hs.sub_globs[s].size(); ++r) dof_subs[hs.sub_globs[s][r]].push_back(s);
    hs.Ac_ptr.assign(nC + 1, 0);
    std::vector<int32_t> where(nC, -1);
    std::vector<int32_t> cols;
    std::vector<double> vals;
    for (int64_t g = 0; g < nC; ++g) {
      cols.clear();
      vals.clear();
      for (int s : dof_subs[g]) {
        const auto& gl = hs.sub_globs[s];
        const int nc = (int)gl.size();
        const int r = (int)(std::lower_bound(gl.begin(), gl.end(), (int32_t)g) - gl.begin());
        for (int c = 0; c < nc; ++c) {
          const int32_t w = gl[c];
          if (where[w] < 0) { where[w] = (int32_t)cols.size(); cols.push_back(w); vals.push_back(0.0); }
          vals[where[w]] += hs.Aci[s][(size_t)r * nc + c];
        }
      }
      std::vector<int> idx(cols.size());
      std::iota(idx.begin(), idx.end(), 0);
      std::sort(idx.begin(), idx.end(), [&](int a, int b) { return cols[a] < cols[b]; });
      for (int i : idx) {
        hs.Ac_col.push_back(cols[i]);
        hs.Ac_val.push_back(vals[i]);
        where[cols[i]] = -1;
      }
      hs.Ac_ptr[g + 1] = (int64_t)hs.Ac_col.size();
    }
    hs.coarse_dense = O->coarse == BDDC_COARSE_DENSE;
    hs.coarse_cg = O->coarse == BDDC_COARSE_CG;
    if (hs.coarse_cg) {
      // the coarse CG works on A_c itself: nothing to factorise
    } else if (factor_coarse && hs.coarse_dense) {
      hs.Acinv.assign((size_t)nC * nC, 0.0);
      for (int64_t r = 0; r < nC; ++r)
        for (int64_t j = hs.Ac_ptr[r]; j < hs.Ac_ptr[r + 1]; ++j) hs.Acinv[(size_t)r * nC + hs.Ac_col[j]] = hs.Ac_val[j];
      if (dense::spd_inverse((int)nC, hs.Acinv.data(), nC, threads) >= 0) {
        err = "coarse matrix A_c is not positive definite";
        return BDDC_ERR_SINGULAR;
      }
    } else if (factor_coarse) {
      // subdomain centroids (element centres, grid units) for the nested dissection
      std::vector<double> sxyz(3 * (size_t)P->n_sub, 0.0);
      std::vector<int64_t> cnt(P->n_sub, 0);
      const int64_t ne = P->ne;
      const int64_t n_el = dim == 3 ? ne * ne * ne : ne * ne;
      for (int64_t e = 0; e < n_el; ++e) {
        const int32_t q = P->elem_subdomain[e];
        sxyz[3 * q] += (double)(e % ne) + 0.5;
        sxyz[3 * q + 1] += (double)((e / ne) % ne) + 0.5;
        sxyz[3 * q + 2] += dim == 3 ? (double)(e / (ne * ne)) + 0.5 : 0.0;
        cnt[q]++;
      }
      for (int32_t q = 0; q < P->n_sub; ++q)
        for (int d = 0; d < 3; ++d) sxyz[3 * q + d] /= (double)std::max<int64_t>(cnt[q], 1);
      const int rc = coarse_factor(nC, hs.Ac_ptr, hs.Ac_col, hs.Ac_val, hs.glob_subs, sxyz, hs.cfac, err,
                                   kCoarseDenseTop);
      if (rc != BDDC_OK) return rc;
    }
  }
  return BDDC_OK;
}

}  // namespace bddc
