// Sparse float64 Cholesky factorisation of the coarse matrix A_c (host side).
//
// The coarse problem A_c u_c = r_c (Sec. 2, Eq. coarsegrid) is solved exactly
// in float64 through a supernodal Cholesky factorisation. Ordering: nested
// dissection of the coarse graph, in which two coarse dofs are adjacent when
// a subdomain holds both, so the graph is a union of one clique per
// subdomain. The dissection therefore splits subdomains, not dofs: the
// current group of subdomains is cut by a plane across the longest extent of
// their centroids (among cuts near the median, the one with the smallest
// separator, lightly penalised for imbalance); a dof all of whose subdomains
// lie on one side goes to that side, a dof with subdomains on both sides is
// in the separator. No subdomain holds dofs of both sides, so this is a
// vertex separator, and it holds only the globs on the surface between the
// two groups (a plane through dofs, by contrast, also takes every far-side
// dof of each subdomain the plane crosses). Every node of the dissection
// tree is a supernode whose pivots are its separator (or, at the leaves, its
// whole vertex set).
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
  const std::vector<std::vector<int32_t>>& subs;   // per dof: its subdomains
  const std::vector<double>& sxyz;                 // per subdomain: centroid
  std::vector<int8_t> side;                        // per subdomain: 1 or 2 during a split
  CoarseFactor& cf;
  std::vector<int32_t> order;                      // position -> dof

  Dissection(const std::vector<std::vector<int32_t>>& s, const std::vector<double>& x, int n_sub, CoarseFactor& f)
      : subs(s), sxyz(x), side(n_sub, 0), cf(f) {}

  // V: the dofs all of whose subdomains are in G. Returns the index of the
  // new tree node (children first).
  int build(std::vector<int32_t> V, std::vector<int32_t> G, int depth) {
    std::vector<int32_t> sep, h1, h2, g1, g2;
    bool leaf = (int)V.size() <= kLeaf || G.size() < 2 || depth > 60;
    if (!leaf) leaf = !split(V, G, sep, h1, h2, g1, g2);
    CoarseNode node;
    std::vector<int> kids;
    if (leaf) {
      node.piv = V;
    } else {
      if (!h1.empty()) kids.push_back(build(std::move(h1), std::move(g1), depth + 1));
      if (!h2.empty()) kids.push_back(build(std::move(h2), std::move(g2), depth + 1));
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

  // 1 or 2: all subdomains of v on that side; 0: on both (separator)
  int dof_side(int32_t v) const {
    int s1 = 0, s2 = 0;
    for (int32_t q : subs[v]) (side[q] == 1 ? s1 : s2)++;
    return s2 == 0 ? 1 : s1 == 0 ? 2 : 0;
  }

  bool split(const std::vector<int32_t>& V, const std::vector<int32_t>& G, std::vector<int32_t>& sep,
             std::vector<int32_t>& h1, std::vector<int32_t>& h2, std::vector<int32_t>& g1,
             std::vector<int32_t>& g2) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t q : G)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], sxyz[3 * q + d]);
        hi[d] = std::max(hi[d], sxyz[3 * q + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    std::vector<int32_t> Gs = G;
    std::stable_sort(Gs.begin(), Gs.end(),
                     [&](int32_t a, int32_t b) { return sxyz[3 * a + ax] < sxyz[3 * b + ax]; });
    // candidate cuts: after position m (first m subdomains on side 1), m in the middle half
    const int ng = (int)Gs.size();
    std::vector<int> cand;
    for (int m = std::max(1, ng / 4); m <= std::min(ng - 1, ng - ng / 4); ++m) cand.push_back(m);
    if (cand.empty()) cand.push_back(ng / 2);
    if (cand.size() > 48) {
      std::vector<int> thin;
      for (size_t i = 0; i < 48; ++i) thin.push_back(cand[i * cand.size() / 48]);
      cand.swap(thin);
    }
    double best_cost = 1e300;
    int best_m = -1;
    for (int m : cand) {
      for (int i = 0; i < ng; ++i) side[Gs[i]] = i < m ? 1 : 2;
      int64_t n1 = 0, n2 = 0, ns = 0;
      for (int32_t v : V) {
        const int sd = dof_side(v);
        (sd == 1 ? n1 : sd == 2 ? n2 : ns)++;
      }
      if (n1 == 0 || n2 == 0) continue;
      const double cost = (double)ns + 0.05 * std::fabs((double)(n1 - n2));
      if (cost < best_cost) { best_cost = cost; best_m = m; }
    }
    if (best_m < 0) return false;
    for (int i = 0; i < ng; ++i) {
      side[Gs[i]] = i < best_m ? 1 : 2;
      (i < best_m ? g1 : g2).push_back(Gs[i]);
    }
    for (int32_t v : V) {
      const int sd = dof_side(v);
      (sd == 1 ? h1 : sd == 2 ? h2 : sep).push_back(v);
    }
    return true;
  }
};

}  // namespace

void coarse_renumber(CoarseFactor& cf, std::vector<int32_t>& perm) {
  perm.assign(cf.n, 0);
  for (int64_t i = 0; i < cf.n; ++i) perm[cf.order[i]] = (int32_t)i;
  for (CoarseNode& T : cf.nodes) {
    for (int32_t& v : T.piv) v = perm[v];
    for (int32_t& w : T.upd) w = perm[w];
  }
  for (int64_t i = 0; i < cf.n; ++i) cf.order[i] = (int32_t)i;
}

int coarse_factor(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& val, const std::vector<std::vector<int32_t>>& dof_subs,
                  const std::vector<double>& sub_xyz, CoarseFactor& cf, std::string& err) {
  cf = CoarseFactor();
  cf.n = n;
  if (n == 0) return BDDC_OK;
  // ---- ordering and tree ----------------------------------------------------------
  const int n_sub = (int)(sub_xyz.size() / 3);
  Dissection nd(dof_subs, sub_xyz, n_sub, cf);
  std::vector<int32_t> all(n), groups(n_sub);
  std::iota(all.begin(), all.end(), 0);
  std::iota(groups.begin(), groups.end(), 0);
  nd.build(std::move(all), std::move(groups), 0);
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
