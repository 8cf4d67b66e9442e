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
#include <thread>
#include <vector>

#include "dense.hpp"
#include "internal.hpp"

namespace bddc {

namespace {

constexpr int kLeaf = 384;  // coarse problem: vertex sets up to this size are not split

struct Dissection {
  const std::vector<std::vector<int32_t>>& subs;   // per dof: its groups (subdomains or elements)
  const std::vector<double>& sxyz;                 // per group: centroid
  std::vector<int8_t> side;                        // per group: 1 or 2 during a split
  CoarseFactor& cf;
  int leaf;                                        // vertex sets up to this size are not split
  std::vector<int32_t> order;                      // position -> dof

  Dissection(const std::vector<std::vector<int32_t>>& s, const std::vector<double>& x, int n_sub, CoarseFactor& f,
             int leaf_size)
      : subs(s), sxyz(x), side(n_sub, 0), cf(f), leaf(leaf_size) {}

  // V: the dofs all of whose subdomains are in G. Returns the index of the
  // new tree node (children first).
  int build(std::vector<int32_t> V, std::vector<int32_t> G, int depth) {
    std::vector<int32_t> sep, h1, h2, g1, g2;
    bool is_leaf = (int)V.size() <= leaf || G.size() < 2 || depth > 60;
    if (!is_leaf) is_leaf = !split(V, G, sep, h1, h2, g1, g2);
    CoarseNode node;
    std::vector<int> kids;
    if (is_leaf) {
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

// Gather form of both sweeps: phases 0 .. L-1 are the forward levels (height
// lv), phases L .. 2L-1 the backward levels (height 2L-1-phase). The
// coefficients and indices of the units of a phase are stored longest unit
// first; for each launch shape the units are assigned to warps longest first,
// each to the warp with the least work so far, and their descriptors stored
// warp by warp.

void gather_layout(const CoarseFactor& cf, int nshapes, const int* blocks, const int* warps_per_block,
                   GatherLayout& g) {
  const int L = cf.n_levels;
  const int nn = (int)cf.nodes.size();
  const int32_t n = (int32_t)cf.n;
  std::vector<int32_t> pos(n), first(nn);
  for (int32_t i = 0; i < n; ++i) pos[cf.order[i]] = i;
  for (int t = 0; t < nn; ++t) first[t] = cf.nodes[t].last - cf.nodes[t].p + 1;
  // kind 0: row i of node a (forward); kind 1: receiving position a with
  // contributions [cb, ce) of rlist; kind 2: row i of node a (backward);
  // kind 3: row a of the dense top's inverse; kind 4: copy of y to u at the
  // dense top's dof a
  struct GU {
    int32_t kind, a, i, len, cb, ce;
  };
  std::vector<int8_t> has(n, 0);   // r' at this position updated by an earlier level
  auto xf = [&](int32_t q) { return has[q] ? q : n + cf.order[q]; };
  std::vector<std::vector<int32_t>> recv(n);
  std::vector<int32_t> touched, rlist, ord;
  std::vector<GU> us;
  std::vector<CGUnit> desc;
  std::vector<double>& gC = g.C;
  std::vector<int32_t>& gI = g.I;
  gC.clear();
  gI.clear();
  g.seq.clear();
  g.seq_off.assign(1, 0);
  // dense top: the levels from height Ht on are one forward-type phase
  // (kind 3: y_T = S_TT^-1 r'_T, row by row); the backward levels below read
  // u_T from y, and the first of them also copies y_T to u (kind 4)
  const int nT = (int)cf.top_pos.size();
  const bool dtop = cf.top_levels > 0 && nT > 0 && (int64_t)cf.top_inv.size() == (int64_t)nT * nT;
  const int Ht = dtop ? L - cf.top_levels : L;
  const int nph = dtop ? 2 * Ht + 1 : 2 * L, nfwd = dtop ? Ht + 1 : L;
  std::vector<int8_t> intop(n, 0);
  if (dtop)
    for (int32_t q : cf.top_pos) intop[q] = 1;
  g.fwd_phases = nfwd;
  g.phases = nph;
  g.units.assign(nshapes, {});
  g.wo.assign(nshapes, {});
  for (int sh = 0; sh < nshapes; ++sh)
    g.wo[sh].assign((size_t)nph * (blocks[sh] * warps_per_block[sh] + 1), 0);
  int64_t total = dtop ? (int64_t)nT * (nT + 1) : 0;
  for (const CoarseNode& T : cf.nodes) total += 2 * (int64_t)T.p * (T.p + T.u);
  gC.reserve((size_t)total);
  gI.reserve((size_t)total);
  std::vector<std::vector<int32_t>> per;
  for (int ph = 0; ph < nph; ++ph) {
    const bool fwd = ph < nfwd;
    const int lv = fwd ? ph : nph - 1 - ph;
    us.clear();
    rlist.clear();
    touched.clear();
    if (dtop && ph == Ht)
      for (int i = 0; i < nT; ++i) us.push_back(GU{3, i, 0, nT, 0, 0});
    if (dtop && !fwd && lv == Ht - 1)
      for (int i = 0; i < nT; ++i) us.push_back(GU{4, i, 0, 1, 0, 0});
    for (int t = 0; t < nn && !(dtop && ph == Ht); ++t) {
      const CoarseNode& T = cf.nodes[t];
      if (T.height != lv || T.p == 0) continue;
      for (int i = 0; i < T.p; ++i) us.push_back(GU{fwd ? 0 : 2, t, i, fwd ? i + 1 : T.p - i + T.u, 0, 0});
      if (!fwd) continue;
      for (int b = 0; b < T.u; ++b) {
        const int32_t w = pos[T.upd[b]];
        if (recv[w].empty()) touched.push_back(w);
        recv[w].push_back(t);
        recv[w].push_back(b);
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int32_t w : touched) {
      const int32_t cb = (int32_t)rlist.size();
      int32_t len = 0;
      for (size_t q = 0; q < recv[w].size(); q += 2) {
        rlist.push_back(recv[w][q]);
        rlist.push_back(recv[w][q + 1]);
        len += cf.nodes[recv[w][q]].p;
      }
      us.push_back(GU{1, w, 0, len, cb, (int32_t)rlist.size()});
      recv[w].clear();
    }
    // coefficients and indices of every unit, longest unit first
    ord.resize(us.size());
    for (size_t k = 0; k < us.size(); ++k) ord[k] = (int32_t)k;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return us[x].len > us[y].len; });
    desc.resize(us.size());
    for (int32_t k : ord) {
      const GU& x = us[k];
      CGUnit d{(int64_t)gC.size(), x.len, 0, -1, 0};
      if (x.kind == 0) {
        const CoarseNode& T = cf.nodes[x.a];
        const int32_t pos0 = first[x.a];
        for (int j = 0; j <= x.i; ++j) {
          gC.push_back(T.Fm[(size_t)x.i * T.p + j]);
          gI.push_back(xf(pos0 + j));
        }
        d.dst = pos0 + x.i;
      } else if (x.kind == 1) {
        for (int32_t q = x.cb; q < x.ce; q += 2) {
          const CoarseNode& T = cf.nodes[rlist[q]];
          const int32_t pos0 = first[rlist[q]], b = rlist[q + 1];
          for (int j = 0; j < T.p; ++j) {
            gC.push_back(T.Fm[(size_t)(T.p + b) * T.p + j]);
            gI.push_back(xf(pos0 + j));
          }
        }
        d.dst = x.a;
        d.aux = xf(x.a);
      } else if (x.kind == 2) {
        const CoarseNode& T = cf.nodes[x.a];
        const int32_t pos0 = first[x.a];
        const size_t f = (size_t)T.p + T.u;
        for (int j = x.i; j < T.p; ++j) {
          gC.push_back(T.Bm[(size_t)x.i * f + j]);
          gI.push_back(pos0 + j);
        }
        for (int b = 0; b < T.u; ++b) {
          const int32_t q = pos[T.upd[b]];
          gC.push_back(T.Bm[(size_t)x.i * f + T.p + b]);
          gI.push_back(intop[q] ? q : n + q);   // u_T is y_T
        }
        d.dst = pos0 + x.i;
        d.aux = cf.order[pos0 + x.i];
      } else if (x.kind == 3) {
        for (int j = 0; j < nT; ++j) {
          gC.push_back(cf.top_inv[(size_t)x.a * nT + j]);
          gI.push_back(xf(cf.top_pos[j]));
        }
        d.dst = cf.top_pos[x.a];
      } else {
        gC.push_back(1.0);
        gI.push_back(cf.top_pos[x.a]);
        d.dst = cf.top_pos[x.a];
        d.aux = cf.order[cf.top_pos[x.a]];
      }
      desc[k] = d;
      g.seq.push_back(d);
    }
    // per launch shape: longest first to the least-loaded warp (cost: batches
    // of kGatherBatch, and a quarter batch per unit for its reduction and store);
    // the h-th least-loaded warp is warp h / blocks of block h % blocks, so
    // the work of a small level spreads over all SMs (their FP64 pipes)
    for (int sh = 0; sh < nshapes; ++sh) {
      const int nb = blocks[sh], wpb = warps_per_block[sh], nw = nb * wpb;
      per.assign(nw, {});
      std::vector<std::pair<int64_t, int32_t>> heap;
      heap.reserve(nw);
      for (int w = 0; w < nw; ++w) heap.emplace_back(0, w);
      auto gt = [](const std::pair<int64_t, int32_t>& x, const std::pair<int64_t, int32_t>& y) { return x > y; };
      for (int32_t k : ord) {
        std::pop_heap(heap.begin(), heap.end(), gt);
        auto& top = heap.back();
        per[top.second].push_back(k);
        top.first += 4 * ((us[k].len + kGatherBatch - 1) / kGatherBatch) + 1;
        std::push_heap(heap.begin(), heap.end(), gt);
      }
      std::vector<CGUnit>& gu = g.units[sh];
      int32_t* wrow = &g.wo[sh][(size_t)ph * (nw + 1)];
      for (int w = 0; w < nw; ++w) {
        wrow[w] = (int32_t)gu.size();
        for (int32_t k : per[(w % wpb) * nb + w / wpb]) gu.push_back(desc[k]);
      }
      wrow[nw] = (int32_t)gu.size();
    }
    g.seq_off.push_back((int64_t)g.seq.size());
    if (fwd)
      for (const GU& x : us)
        if (x.kind == 1) has[x.a] = 1;
  }
}

int sparse_factor(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& val, const std::vector<std::vector<int32_t>>& dof_groups,
                  const std::vector<double>& group_xyz, int64_t n_keep, int leaf, CoarseFactor& cf,
                  std::vector<double>* schur, std::string& err, int64_t top_max) {
  cf = CoarseFactor();
  cf.n = n;
  const int64_t nf = n - n_keep;        // dofs eliminated
  if (n == 0) return BDDC_OK;
  // ---- ordering and tree ----------------------------------------------------------
  // the dissection orders the dofs [0, nf); the kept dofs [nf, n) form one
  // last front above it (its root), assembled but not factorised
  const int n_groups = (int)(group_xyz.size() / 3);
  Dissection nd(dof_groups, group_xyz, n_groups, cf, std::max(1, leaf));
  int top = -1;
  if (nf > 0) {
    std::vector<int32_t> all(nf), groups(n_groups);
    std::iota(all.begin(), all.end(), 0);
    std::iota(groups.begin(), groups.end(), 0);
    top = nd.build(std::move(all), std::move(groups), 0);
  }
  if (n_keep > 0) {
    CoarseNode root;
    for (int64_t v = nf; v < n; ++v) root.piv.push_back((int32_t)v);
    if (top >= 0) root.children.push_back(top);
    root.first = top >= 0 ? cf.nodes[top].first : 0;
    for (int32_t v : root.piv) nd.order.push_back(v);
    root.last = (int)n - 1;
    cf.nodes.push_back(std::move(root));
    if (top >= 0) cf.nodes[top].parent = (int)cf.nodes.size() - 1;
  }
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

  // ---- dense top: the most top levels with at most top_max dofs --------------------
  // (T: the pivots of the nodes of height >= Ht; its Schur complement S
  // collects A_TT and the update matrices of the nodes below T whose
  // parents are in T)
  int Ht = -1, nT = 0;
  std::vector<int32_t> tidx;
  std::vector<double> S;
  if (top_max > 0 && n_keep == 0 && cf.n_levels >= 2) {
    std::vector<int64_t> ph(cf.n_levels, 0);
    for (const CoarseNode& T : cf.nodes) ph[T.height] += T.p;
    int64_t cum = 0;
    for (int h = cf.n_levels - 1; h >= 1; --h) {
      if (cum + ph[h] > top_max) break;
      cum += ph[h];
      Ht = h;
    }
  }
  if (Ht >= 1) {
    for (const CoarseNode& T : cf.nodes)
      if (T.height >= Ht)
        for (int32_t v : T.piv) cf.top_pos.push_back(pos[v]);
    std::sort(cf.top_pos.begin(), cf.top_pos.end());
    nT = (int)cf.top_pos.size();
    tidx.assign(n, -1);
    for (int i = 0; i < nT; ++i) tidx[cf.order[cf.top_pos[i]]] = i;
    S.assign((size_t)nT * nT, 0.0);
    cf.top_levels = cf.n_levels - Ht;
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
      if (Ht >= 1 && T.height >= Ht && K.height < Ht)
        for (int a = 0; a < K.u; ++a) {
          const size_t ra = (size_t)tidx[K.upd[a]] * nT;
          for (int b = 0; b < K.u; ++b) S[ra + tidx[K.upd[b]]] += Uk[(size_t)a * K.u + b];
        }
      std::vector<double>().swap(upd_mat[k]);
    }
    for (int i = 0; i < p; ++i) loc[T.piv[i]] = -1;
    for (int i = 0; i < u; ++i) loc[T.upd[i]] = -1;
    if (n_keep > 0 && t == nn - 1) {
      // the kept dofs' front is their Schur complement (pivots ascending, u = 0)
      if (schur) *schur = std::move(F);
      break;
    }
    T.Fm.assign((size_t)f * p, 0.0);
    T.Bm.assign((size_t)p * f, 0.0);
    if (p > 0) {
      // L_PP and its inverse
      std::vector<double> L((size_t)p * p), Li((size_t)p * p), Ai((size_t)p * p);
      for (int i = 0; i < p; ++i) std::memcpy(&L[(size_t)i * p], &F[(size_t)i * f], sizeof(double) * p);
      if (dense::potrf(p, L.data(), p) >= 0) {
        err = n_keep > 0 ? "a local interior matrix A_II is not positive definite"
                         : "coarse matrix A_c is not positive definite";
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
  if (Ht >= 1) {
    // S_TT = A_TT + (the update matrices gathered above); its inverse is (A^-1)_TT
    for (int i = 0; i < nT; ++i) {
      const int32_t v = cf.order[cf.top_pos[i]];
      for (int64_t j = rp[v]; j < rp[v + 1]; ++j)
        if (tidx[ci[j]] >= 0) S[(size_t)i * nT + tidx[ci[j]]] += val[j];
    }
    for (int i = 0; i < nT; ++i)
      for (int j = i + 1; j < nT; ++j) {
        const double m = 0.5 * (S[(size_t)i * nT + j] + S[(size_t)j * nT + i]);
        S[(size_t)i * nT + j] = S[(size_t)j * nT + i] = m;
      }
    const int threads = (int)std::max(1u, std::thread::hardware_concurrency());
    if (dense::spd_inverse(nT, S.data(), nT, threads) >= 0) {
      err = "the Schur complement of the coarse factor's top levels is not positive definite";
      return BDDC_ERR_SINGULAR;
    }
    cf.top_inv = std::move(S);
  }
  if (n_keep > 0) {
    // drop the kept front and the kept dofs from every update set (a suffix:
    // update sets are in elimination order and the kept dofs come last), with
    // their rows of Fm and columns of Bm: what remains factorises A_FF alone
    cf.nodes.pop_back();
    if (top >= 0) cf.nodes[top].parent = -1;
    cf.n = nf;
    cf.order.resize(nf);
    cf.nnz = 0;
    cf.n_levels = 0;
    for (CoarseNode& T : cf.nodes) {
      int u2 = 0;
      while (u2 < T.u && T.upd[u2] < nf) ++u2;
      if (u2 < T.u) {
        const int p = T.p, f = p + T.u, f2 = p + u2;
        T.Fm.resize((size_t)f2 * p);
        std::vector<double> B2((size_t)p * f2);
        for (int i = 0; i < p; ++i) std::memcpy(&B2[(size_t)i * f2], &T.Bm[(size_t)i * f], sizeof(double) * f2);
        T.Bm.swap(B2);
        T.upd.resize(u2);
        T.u = u2;
      }
      cf.nnz += (int64_t)(T.p + T.u) * T.p;
      cf.n_levels = std::max(cf.n_levels, T.height + 1);
    }
  }
  return BDDC_OK;
}

void level_phases(const GatherLayout& g, std::vector<SweepSet::LevelPhase>& out) {
  out.clear();
  for (size_t ph = 0; ph + 1 < g.seq_off.size(); ++ph) {
    SweepSet::LevelPhase P{};
    P.u0 = g.seq_off[ph];
    const int32_t m = (int32_t)(g.seq_off[ph + 1] - g.seq_off[ph]);
    int32_t k = 0;
    for (int c = 0; c < kLevelClasses; ++c) {
      P.cb[c] = k;
      while (k < m && level_class(g.seq[P.u0 + k].len) <= c) ++k;
    }
    P.cb[kLevelClasses] = m;
    P.bb[0] = 0;
    for (int c = 0; c < kLevelClasses; ++c) {
      const int per = kLevelThreads / kLevelGroup[c];
      P.bb[c + 1] = P.bb[c] + (P.cb[c + 1] - P.cb[c] + per - 1) / per;
    }
    out.push_back(P);
  }
}

void block_layout(const CoarseFactor& cf, int64_t target, BlockLayout& out) {
  out = BlockLayout();
  const int nn = (int)cf.nodes.size(), L = cf.n_levels;
  out.nodes.resize(nn);
  int64_t fcur = 0, bcur = 0, ccur = 0;
  for (int t = 0; t < nn; ++t) {
    const CoarseNode& T = cf.nodes[t];
    SNode& d = out.nodes[t];
    d.p = T.p;
    d.u = T.u;
    d.pos0 = T.last - T.p + 1;
    d.fld = std::max(T.p, 1);
    d.bld = std::max(T.p + T.u, 1);
    fcur = (fcur + 31) / 32 * 32;   // the layout of the several-column node matrices
    d.foff = fcur;
    fcur += (int64_t)(T.p + T.u) * d.fld;
    bcur = (bcur + 31) / 32 * 32;
    d.boff = bcur;
    bcur += (int64_t)T.p * d.bld;
    d.cbase = (int32_t)ccur;
    ccur += T.u;
    d.cmap0 = 0;
    d.upd_off = (int32_t)out.upd.size();
    out.upd.insert(out.upd.end(), T.upd.begin(), T.upd.end());
    d.kid0 = (int32_t)out.kids.size();
    d.nkid = (int32_t)T.children.size();
    d.height = T.height;
    out.kids.insert(out.kids.end(), T.children.begin(), T.children.end());
    out.max_front = std::max(out.max_front, T.p + T.u);
  }
  out.cbuf = ccur;
  // each child's update set as indices into its parent's front: the
  // parent's pivots (contiguous positions), then its update set
  std::vector<int32_t> where(cf.n, -1);
  for (int q = 0; q < nn; ++q) {
    const CoarseNode& Q = cf.nodes[q];
    if (Q.children.empty()) continue;
    const SNode& dq = out.nodes[q];
    for (int i = 0; i < Q.p; ++i) where[dq.pos0 + i] = i;
    for (int b = 0; b < Q.u; ++b) where[Q.upd[b]] = Q.p + b;
    for (int k : Q.children) {
      out.nodes[k].cmap0 = (int32_t)out.cmap.size();
      for (int32_t w : cf.nodes[k].upd) out.cmap.push_back(where[w]);
    }
    for (int i = 0; i < Q.p; ++i) where[dq.pos0 + i] = -1;
    for (int b = 0; b < Q.u; ++b) where[Q.upd[b]] = -1;
  }
  out.F.assign((size_t)std::max<int64_t>(fcur, 1), 0.0);
  out.B.assign((size_t)std::max<int64_t>(bcur, 1), 0.0);
  for (int t = 0; t < nn; ++t) {
    const CoarseNode& T = cf.nodes[t];
    const SNode& d = out.nodes[t];
    const int f = T.p + T.u;
    for (int r = 0; r < f && T.p > 0; ++r)
      std::memcpy(&out.F[d.foff + (int64_t)r * d.fld], &T.Fm[(size_t)r * T.p], sizeof(double) * T.p);
    for (int r = 0; r < T.p; ++r)
      std::memcpy(&out.B[d.boff + (int64_t)r * d.bld], &T.Bm[(size_t)r * f], sizeof(double) * f);
  }
  // work items: chunks of rows, largest chunks of a phase first
  out.item_off.assign(1, 0);
  std::vector<BlockItem> small;
  auto chunks = [&](int t, int rows, int len) {
    const SNode& d = out.nodes[t];
    if (d.p + d.u <= kSmallFront) {
      small.push_back(BlockItem{t, 0, rows, block_group(len)});
      return;
    }
    const int64_t per = std::max<int64_t>(1, target / std::max(len, 1));
    const int R = (int)std::min<int64_t>(rows, std::max<int64_t>(8, per));
    for (int r0 = 0; r0 < rows; r0 += R)
      out.items.push_back(BlockItem{t, r0, std::min(R, rows - r0), block_group(len)});
  };
  auto close_phase = [&](bool fwd) {
    auto work = [&](const BlockItem& x) {
      const SNode& a = out.nodes[x.node];
      return (int64_t)x.nrows * (fwd ? a.p : a.p + a.u);
    };
    auto heavier = [&](const BlockItem& x, const BlockItem& y) { return work(x) > work(y); };
    const int64_t b = out.item_off.back();
    std::stable_sort(out.items.begin() + b, out.items.end(), heavier);
    out.n_big.push_back((int64_t)out.items.size() - b);
    std::stable_sort(small.begin(), small.end(), heavier);
    out.items.insert(out.items.end(), small.begin(), small.end());
    small.clear();
    out.item_off.push_back((int64_t)out.items.size());
  };
  for (int lv = 0; lv < L; ++lv) {
    for (int t = 0; t < nn; ++t) {
      const CoarseNode& T = cf.nodes[t];
      if (T.height == lv && T.p + T.u > 0) chunks(t, T.p + T.u, T.p);
    }
    close_phase(true);
  }
  for (int lv = L - 1; lv >= 0; --lv) {
    for (int t = 0; t < nn; ++t) {
      const CoarseNode& T = cf.nodes[t];
      if (T.height == lv && T.p > 0) chunks(t, T.p, T.p + T.u);
    }
    close_phase(false);
  }
}

int coarse_factor(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& val, const std::vector<std::vector<int32_t>>& dof_subs,
                  const std::vector<double>& sub_xyz, CoarseFactor& cf, std::string& err, int64_t top_max) {
  return sparse_factor(n, rp, ci, val, dof_subs, sub_xyz, 0, kLeaf, cf, nullptr, err, top_max);
}

void merge_forest(const std::vector<CoarseFactor>& parts, const std::vector<int32_t>& off, CoarseFactor& out) {
  out = CoarseFactor();
  int64_t n = 0;
  for (size_t s = 0; s < parts.size(); ++s) n = std::max<int64_t>(n, off[s] + parts[s].n);
  out.n = n;
  out.order.assign(n, 0);
  for (size_t s = 0; s < parts.size(); ++s) {
    const CoarseFactor& P = parts[s];
    const int32_t o = off[s];
    const int t0 = (int)out.nodes.size();
    for (int64_t i = 0; i < P.n; ++i) out.order[o + i] = o + P.order[i];
    for (const CoarseNode& T : P.nodes) {
      CoarseNode N = T;
      for (int32_t& v : N.piv) v += o;
      for (int32_t& w : N.upd) w += o;
      for (int& k : N.children) k += t0;
      if (N.parent >= 0) N.parent += t0;
      N.first += o;
      N.last += o;
      out.nodes.push_back(std::move(N));
    }
    out.n_levels = std::max(out.n_levels, P.n_levels);
    out.nnz += P.nnz;
  }
}

}  // namespace bddc
