// Sparse float64 Cholesky factorisation of the coarse matrix A_c (host side).
//
// The coarse problem A_c u_c = r_c (Sec. 2, Eq. coarsegrid) is solved exactly
// in float64 through a supernodal Cholesky factorisation. Ordering: nested
// dissection of the coarse graph (two coarse dofs are adjacent when a
// subdomain holds both), by recursive geometric bisection of the globs'
// centroids. Among cut planes near the median, the one whose vertex
// separator (dofs on the far side with a neighbour on the near side) is
// smallest is taken. Every node of the dissection tree is a supernode whose
// pivots are its separator (or, at the leaves, its whole vertex set).
//
// Factorisation: multifrontal. The front of node t holds its pivots P and
// its update set U (the later dofs coupled to t's subtree). With
// L_PP L_PP^T = F_PP (dense Cholesky), the node stores
//   Fm = [L_PP^-1 ; M]        ((p+u) x p, forward sweep),   M = L_UP L_PP^-1
//   Bm = [L_PP^-T , -M^T]     (p x (p+u), backward sweep)
// so that the forward step is  y_P = L_PP^-1 r'_P,  c = M r'_P  and the
// backward step is  u_P = L_PP^-T y_P - M^T u_U: each one dense product,
// which the GPU applies level by level. The update matrix passed to the
// parent is F_UU - M F_PU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "dense.hpp"
#include "internal.hpp"

namespace bddc {

namespace {

constexpr int kLeaf = 384;  // vertex sets up to this size are not split

struct Dissection {
  const std::vector<int64_t>& rp;
  const std::vector<int32_t>& ci;
  const std::vector<double>& xyz;
  std::vector<int32_t> stamp;       // per dof: id of the set it currently belongs to
  std::vector<double> cpos;         // per dof: coordinate along the current axis
  int next_stamp = 1;
  CoarseFactor& cf;
  std::vector<int32_t> order;       // position -> dof

  Dissection(const std::vector<int64_t>& r, const std::vector<int32_t>& c, const std::vector<double>& x,
             int64_t n, CoarseFactor& f)
      : rp(r), ci(c), xyz(x), stamp(n, 0), cpos(n, 0.0), cf(f) {}

  // Split V; returns the index of the new tree node (children first).
  int build(std::vector<int32_t> V, int depth) {
    std::vector<int32_t> sep, h1, h2;
    bool leaf = (int)V.size() <= kLeaf || depth > 60;
    if (!leaf) leaf = !split(V, sep, h1, h2);
    CoarseNode node;
    std::vector<int> kids;
    if (leaf) {
      node.piv = V;
    } else {
      if (!h1.empty()) kids.push_back(build(std::move(h1), depth + 1));
      if (!h2.empty()) kids.push_back(build(std::move(h2), depth + 1));
      node.piv = sep;
    }
    std::sort(node.piv.begin(), node.piv.end());
    node.children = kids;
    node.first = kids.empty() ? (int)order.size() : cf.nodes[kids.front()].first;
    for (int32_t v : node.piv) order.push_back(v);
    node.last = (int)order.size() - 1;
    cf.nodes.push_back(std::move(node));
    const int id = (int)cf.nodes.size() - 1;
    for (int k : kids) cf.nodes[k].parent = id;
    return id;
  }

  bool split(const std::vector<int32_t>& V, std::vector<int32_t>& sep, std::vector<int32_t>& h1,
             std::vector<int32_t>& h2) {
    // axis of largest extent
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t v : V)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xyz[3 * v + d]);
        hi[d] = std::max(hi[d], xyz[3 * v + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    if (!(hi[ax] > lo[ax])) return false;
    std::vector<double> c(V.size());
    for (size_t i = 0; i < V.size(); ++i) c[i] = xyz[3 * V[i] + ax];
    std::vector<double> sc = c;
    std::sort(sc.begin(), sc.end());
    // candidate cut values: distinct coordinates in the middle half
    std::vector<double> cand;
    const size_t a = sc.size() / 4, b = sc.size() - sc.size() / 4;
    for (size_t i = std::max<size_t>(a, 1); i < b; ++i)
      if (sc[i] > sc[i - 1]) cand.push_back(sc[i]);
    if (cand.empty())
      for (size_t i = 1; i < sc.size(); ++i)
        if (sc[i] > sc[i - 1]) cand.push_back(sc[i]);
    if (cand.empty()) return false;
    if (cand.size() > 48) {
      std::vector<double> thin;
      for (size_t i = 0; i < 48; ++i) thin.push_back(cand[i * cand.size() / 48]);
      cand.swap(thin);
    }
    const int st = next_stamp++;
    for (int32_t v : V) stamp[v] = st;
    for (size_t i = 0; i < V.size(); ++i) cpos[V[i]] = c[i];
    double best_cost = 1e300, best_s = 0;
    for (double s : cand) {
      int64_t n1 = 0, ns = 0;
      for (size_t i = 0; i < V.size(); ++i) {
        if (c[i] < s) { ++n1; continue; }
        const int32_t v = V[i];
        for (int64_t j = rp[v]; j < rp[v + 1]; ++j) {
          const int32_t w = ci[j];
          if (stamp[w] == st && cpos[w] < s) { ++ns; break; }
        }
      }
      const int64_t n2 = (int64_t)V.size() - n1 - ns;
      if (n1 == 0 || n2 <= 0) continue;
      const double cost = (double)ns + 0.05 * std::fabs((double)(n1 - n2));
      if (cost < best_cost) { best_cost = cost; best_s = s; }
    }
    if (best_cost >= 1e299) return false;
    for (size_t i = 0; i < V.size(); ++i) {
      const int32_t v = V[i];
      if (c[i] < best_s) { h1.push_back(v); continue; }
      bool touches = false;
      for (int64_t j = rp[v]; j < rp[v + 1] && !touches; ++j) {
        const int32_t w = ci[j];
        touches = stamp[w] == st && cpos[w] < best_s;
      }
      (touches ? sep : h2).push_back(v);
    }
    return !sep.empty() || (!h1.empty() && !h2.empty());
  }
};

}  // namespace

int coarse_factor(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& val, const std::vector<double>& xyz, CoarseFactor& cf,
                  std::string& err) {
  cf = CoarseFactor();
  cf.n = n;
  if (n == 0) return BDDC_OK;
  // ---- ordering and tree ----------------------------------------------------------
  Dissection nd(rp, ci, xyz, n, cf);
  std::vector<int32_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  nd.build(std::move(all), 0);
  std::vector<int32_t> pos(n);
  for (int64_t i = 0; i < n; ++i) pos[nd.order[i]] = (int32_t)i;
  cf.order = nd.order;
  const int nn = (int)cf.nodes.size();   // nodes are in post-order (children before parents)

  // ---- symbolic: update sets --------------------------------------------------------
  std::vector<int32_t> mark(n, -1);
  for (int t = 0; t < nn; ++t) {
    CoarseNode& nd_t = cf.nodes[t];
    std::vector<int32_t> upd;
    auto add = [&](int32_t w) {
      if (pos[w] > nd_t.last && mark[w] != t) { mark[w] = t; upd.push_back(w); }
    };
    for (int32_t v : nd_t.piv)
      for (int64_t j = rp[v]; j < rp[v + 1]; ++j) add(ci[j]);
    for (int k : nd_t.children)
      for (int32_t w : cf.nodes[k].upd) add(w);
    std::sort(upd.begin(), upd.end(), [&](int32_t a, int32_t b) { return pos[a] < pos[b]; });
    nd_t.upd = std::move(upd);
    nd_t.p = (int)nd_t.piv.size();
    nd_t.u = (int)nd_t.upd.size();
    int hgt = 0;
    for (int k : nd_t.children) hgt = std::max(hgt, cf.nodes[k].height + 1);
    nd_t.height = hgt;
    cf.n_levels = std::max(cf.n_levels, hgt + 1);
  }

  // ---- numeric: multifrontal ------------------------------------------------------------
  std::vector<int32_t> loc(n, -1);
  std::vector<std::vector<double>> upd_mat(nn);
  for (int t = 0; t < nn; ++t) {
    CoarseNode& T = cf.nodes[t];
    const int p = T.p, u = T.u, f = p + u;
    for (int i = 0; i < p; ++i) loc[T.piv[i]] = i;
    for (int i = 0; i < u; ++i) loc[T.upd[i]] = p + i;
    std::vector<double> F((size_t)f * f, 0.0);
    // original entries in the pivot rows and columns
    for (int i = 0; i < p; ++i) {
      const int32_t v = T.piv[i];
      for (int64_t j = rp[v]; j < rp[v + 1]; ++j) {
        const int32_t w = ci[j];
        const int lw = loc[w];
        if (lw < 0 || pos[w] < T.first) continue;
        if (lw < p) {
          F[(size_t)i * f + lw] += val[j];
        } else {
          F[(size_t)i * f + lw] += val[j];
          F[(size_t)lw * f + i] += val[j];
        }
      }
    }
    // extend-add of the children's update matrices
    for (int k : T.children) {
      const CoarseNode& K = cf.nodes[k];
      const std::vector<double>& Uk = upd_mat[k];
      for (int a = 0; a < K.u; ++a) {
        const int la = loc[K.upd[a]];
        for (int b = 0; b < K.u; ++b) F[(size_t)la * f + loc[K.upd[b]]] += Uk[(size_t)a * K.u + b];
      }
      std::vector<double>().swap(upd_mat[k]);
    }
    for (int i = 0; i < p; ++i) loc[T.piv[i]] = -1;
    for (int i = 0; i < u; ++i) loc[T.upd[i]] = -1;
    T.Fm.assign((size_t)f * p, 0.0);
    T.Bm.assign((size_t)p * f, 0.0);
    if (p > 0) {
      // L_PP and its inverse
      std::vector<double> L((size_t)p * p), Li((size_t)p * p), Ai((size_t)p * p);
      for (int i = 0; i < p; ++i) std::memcpy(&L[(size_t)i * p], &F[(size_t)i * f], sizeof(double) * p);
      if (dense::potrf(p, L.data(), p) >= 0) {
        err = "coarse matrix A_c is not positive definite";
        return BDDC_ERR_SINGULAR;
      }
      dense::trtri_lower(p, L.data(), p, Li.data(), p);
      dense::lower_gram(p, Li.data(), p, Ai.data(), p);           // F_PP^-1
      for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
          T.Fm[(size_t)i * p + j] = Li[(size_t)i * p + j];          // L_PP^-1
          T.Bm[(size_t)i * f + j] = Li[(size_t)j * p + i];          // L_PP^-T
        }
      if (u > 0) {
        // M = L_UP L_PP^-1 = F_UP F_PP^-1 ; update = F_UU - M F_PU
        std::vector<double> M((size_t)u * p, 0.0);
        dense::gemm_nn(u, p, p, 1.0, &F[(size_t)p * f], f, Ai.data(), p, M.data(), p);
        std::vector<double> Up((size_t)u * u);
        for (int a = 0; a < u; ++a)
          std::memcpy(&Up[(size_t)a * u], &F[(size_t)(p + a) * f + p], sizeof(double) * u);
        dense::gemm_nn(u, u, p, -1.0, M.data(), p, &F[p], f, Up.data(), u);
        for (int a = 0; a < u; ++a)
          for (int b = a + 1; b < u; ++b) {
            const double m = 0.5 * (Up[(size_t)a * u + b] + Up[(size_t)b * u + a]);
            Up[(size_t)a * u + b] = Up[(size_t)b * u + a] = m;
          }
        upd_mat[t] = std::move(Up);
        for (int a = 0; a < u; ++a)
          for (int j = 0; j < p; ++j) {
            T.Fm[(size_t)(p + a) * p + j] = M[(size_t)a * p + j];
            T.Bm[(size_t)j * f + p + a] = -M[(size_t)a * p + j];
          }
      }
    } else if (u > 0) {
      upd_mat[t].assign((size_t)u * u, 0.0);
      for (int a = 0; a < u; ++a)
        std::memcpy(&upd_mat[t][(size_t)a * u], &F[(size_t)a * f], sizeof(double) * u);
    }
    cf.nnz += (int64_t)f * p;
  }
  return BDDC_OK;
}

}  // namespace bddc
