// Host check of the gather form of the factor sweeps (test helper, built and
// run by test_coarse_layout_host.py). Two modes.
//
// coarse ne nsub jitter blocks:wpb ...: sets up a 3D problem through the
// library's host setup, renumbers the coarse factor by elimination order,
// builds the gather layout for the given launch shapes, and emulates the
// sweeps phase by phase, warp by warp, unit by unit, as the kernel reads and
// writes them. Checks: every descriptor and index in range; within a phase
// no value read that the phase writes (except a receiving dof's own value);
// every position's y and u written exactly once; the result solves
// A_c u = r to 1e-12; and all shapes give bitwise the same u.
//
// local dim ne nsub jitter leaf blocks:wpb ...: the sparse local solver.
// Sets the problem up twice, with the dense and with the sparse local
// solver, and checks per subdomain that the couplings A_GI, A_IG are the
// same and that K_GG, Phi_G and A_ci agree to 1e-10 (the Schur complement
// from the partial factorisation against the dense one); then merges the
// interior factors into one forest as the device does (each renumbered by
// elimination order), emulates its gather-form sweeps as above, and checks
// the result against the dense A_II^-1 r of every subdomain to 1e-10; and
// checks the per-level form (class ranges and block counts of every phase;
// the sweeps with each phase's units in storage order give bitwise the same
// result) and the block form (supernode by supernode: fronts from the
// children's contribution vectors, chunks of rows; every row covered once,
// nothing read before the phase that writes it) against the dense solves.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <set>
#include <string>
#include <vector>

#include "../paper_2410_14786_gb300/csrc/internal.hpp"

using namespace bddc;

namespace {

// Emulates the gather-form sweeps of launch shape sh (nw warps) on r (dof
// order, elimination-order numbering); u receives the result. Returns the
// number of failed structural checks.
int emulate(const CoarseFactor& cf, const GatherLayout& gl, int sh, int nw, const std::vector<double>& r,
            std::vector<double>& u, const char* what) {
  const int n = (int)cf.n, NF = gl.fwd_phases, NP = gl.phases;
  int bad = 0;
  if (NP != (cf.top_levels ? 2 * (cf.n_levels - cf.top_levels) + 1 : 2 * cf.n_levels) ||
      NF != (cf.top_levels ? cf.n_levels - cf.top_levels + 1 : cf.n_levels))
    ++bad;
  for (int32_t ix : gl.I)
    if (ix < 0 || ix >= 2 * n) ++bad;
  const std::vector<CGUnit>& U = gl.units[sh];
  const std::vector<int32_t>& wo = gl.wo[sh];
  if (wo.size() != (size_t)NP * (nw + 1) || wo.front() != 0 || wo.back() != (int)U.size()) ++bad;
  for (size_t i = 1; i < wo.size(); ++i)
    if (wo[i] < wo[i - 1]) ++bad;
  for (const CGUnit& d : U)
    if (d.off < 0 || d.len < 1 || d.off + d.len > (int64_t)gl.C.size() || d.dst < 0 || d.dst >= n) ++bad;
  const double nan = std::nan("");
  std::vector<double> rp(n, nan), y(n, nan);
  u.assign(n, nan);
  std::vector<int> ny(n, 0), nu(n, 0);
  int races = 0, nanreads = 0;
  for (int ph = 0; ph < NP; ++ph) {
    const bool fwd = ph < NF;
    std::vector<std::pair<int, double>> wrp, wy, wu;
    std::set<int> rd_rp, rd_y;
    for (int w = 0; w < nw; ++w)
      for (int k = wo[(size_t)ph * (nw + 1) + w]; k < wo[(size_t)ph * (nw + 1) + w + 1]; ++k) {
        const CGUnit& d = U[k];
        auto X = [&](int ix) {
          double v;
          if (fwd) {
            if (ix < n) { v = rp[ix]; rd_rp.insert(ix); } else v = r[ix - n];
          } else {
            if (ix < n) { v = y[ix]; rd_y.insert(ix); } else { v = rp[ix - n]; rd_rp.insert(ix - n); }
          }
          if (std::isnan(v)) ++nanreads;
          return v;
        };
        double s = 0;
        for (int j = 0; j < d.len; ++j) s += gl.C[d.off + j] * X(gl.I[d.off + j]);
        if (!fwd) {
          wrp.push_back({d.dst, s});
          wu.push_back({d.aux, s});
        } else if (d.aux < 0) {
          wy.push_back({d.dst, s});
        } else {
          const double x0 = X(d.aux);
          if (d.aux < n) rd_rp.erase(d.aux);
          wrp.push_back({d.dst, x0 - s});
        }
      }
    std::set<int> seen;
    for (auto& p : wrp) {
      if (rd_rp.count(p.first) || !seen.insert(p.first).second) ++races;
      rp[p.first] = p.second;
    }
    for (auto& p : wy) {
      if (rd_y.count(p.first)) ++races;
      y[p.first] = p.second;
      ++ny[p.first];
    }
    for (auto& p : wu) {
      u[p.first] = p.second;
      ++nu[p.first];
    }
  }
  int once = 0;
  for (int i = 0; i < n; ++i)
    if (ny[i] != 1 || nu[i] != 1) ++once;
  printf("%s shape %d warps: n %d phases %d (dense top of %d levels, %zu dofs) races %d nan-reads %d write-count %d\n",
         what, nw, n, NP, cf.top_levels, cf.top_pos.size(), races, nanreads, once);
  return bad + races + nanreads + once;
}

// Emulates the one-column sweeps as the block form runs them with split
// height kmin: heights below kmin as per-level gather phases (gl.seq; r'
// starts as a copy of r; backward operands u by position), heights from kmin
// on supernode by supernode (fronts from r' and the children from kmin on);
// each phase's writes applied at its end, as the next launch sees them. r in
// positions; u receives the result. Returns the number of failed checks
// (indices out of range, rows not covered exactly once, reads of values not
// yet written).
int emulate_block(const CoarseFactor& cf, const BlockLayout& bl, const GatherLayout& gl, int kmin,
                  const std::vector<double>& r, std::vector<double>& u) {
  const int n = (int)cf.n, L = cf.n_levels;
  const double nan = std::nan("");
  std::vector<double> y(n, nan), cb(bl.cbuf, nan), rp(n, nan);
  if (kmin > 0) rp = r;
  u.assign(n, nan);
  int bad = 0, nanreads = 0;
  std::vector<int> fcover(bl.nodes.size(), 0), bcover(bl.nodes.size(), 0);
  if (bl.item_off.size() != (size_t)2 * L + 1 || bl.item_off.back() != (int64_t)bl.items.size() ||
      bl.n_big.size() != (size_t)2 * L || gl.seq_off.size() != (size_t)2 * L + 1)
    ++bad;
  // a phase's first n_big items are chunks of nodes with fronts above
  // kSmallFront, the rest whole nodes with fronts up to it
  for (int ph = 0; ph < 2 * L && !bad; ++ph)
    for (int64_t k = bl.item_off[ph]; k < bl.item_off[ph + 1]; ++k) {
      const SNode& d = bl.nodes[bl.items[k].node];
      const bool big = k < bl.item_off[ph] + bl.n_big[ph];
      if (big != (d.p + d.u > kSmallFront)) ++bad;
      if (!big && (bl.items[k].row0 != 0 || bl.items[k].nrows != (ph < L ? d.p + d.u : d.p))) ++bad;
      if (d.height != (ph < L ? ph : 2 * L - 1 - ph)) ++bad;
    }
  for (int ph = 0; ph < 2 * L && !bad; ++ph) {
    const bool fwd = ph < L;
    const int height = fwd ? ph : 2 * L - 1 - ph;
    std::vector<std::pair<int64_t, double>> wy, wc, wu, wrp;
    if (height < kmin) {
      // gather phase
      for (int64_t k = gl.seq_off[ph]; k < gl.seq_off[ph + 1]; ++k) {
        const CGUnit& d = gl.seq[k];
        auto X = [&](int ix) {
          const double v = fwd ? (ix < n ? rp[ix] : r[ix - n]) : (ix < n ? y[ix] : u[ix - n]);
          if (std::isnan(v)) ++nanreads;
          return v;
        };
        double sum = 0;
        for (int j = 0; j < d.len; ++j) sum += gl.C[d.off + j] * X(gl.I[d.off + j]);
        if (!fwd) {
          wrp.push_back({d.dst, sum});
          wu.push_back({d.aux, sum});
        } else if (d.aux < 0) {
          wy.push_back({d.dst, sum});
        } else {
          wrp.push_back({d.dst, X(d.aux) - sum});
        }
      }
    } else {
      for (int64_t k = bl.item_off[ph]; k < bl.item_off[ph + 1]; ++k) {
        const BlockItem& it = bl.items[k];
        const SNode& d = bl.nodes[it.node];
        const int f = d.p + d.u;
        if (it.g != 4 && it.g != 8 && it.g != 16 && it.g != 32) ++bad;
        if (it.row0 < 0 || it.nrows < 1 || it.row0 + it.nrows > (fwd ? f : d.p)) { ++bad; continue; }
        (fwd ? fcover : bcover)[it.node] += it.nrows;
        std::vector<double> v(f, 0.0);
        if (fwd) {
          for (int i = 0; i < d.p; ++i) {
            v[i] = kmin > 0 ? rp[d.pos0 + i] : r[d.pos0 + i];
            if (std::isnan(v[i])) ++nanreads;
          }
          for (int q = 0; q < d.nkid; ++q) {
            const SNode& kd = bl.nodes[bl.kids[d.kid0 + q]];
            if (kd.height < kmin) continue;
            for (int a = 0; a < kd.u; ++a) {
              const int32_t w = bl.cmap[kd.cmap0 + a];
              const double c = cb[kd.cbase + a];
              if (w < 0 || w >= f) { ++bad; continue; }
              if (std::isnan(c)) ++nanreads;
              v[w] += c;
            }
          }
          for (int row = it.row0; row < it.row0 + it.nrows; ++row) {
            const int len = row < d.p ? row + 1 : d.p;
            double sum = 0;
            for (int j = 0; j < len; ++j) sum += bl.F[d.foff + (int64_t)row * d.fld + j] * v[j];
            if (row < d.p) wy.push_back({d.pos0 + row, sum});
            else wc.push_back({d.cbase + row - d.p, v[row] - sum});
          }
        } else {
          for (int i = 0; i < d.p; ++i) {
            v[i] = y[d.pos0 + i];
            if (std::isnan(v[i])) ++nanreads;
          }
          for (int b2 = 0; b2 < d.u; ++b2) {
            const int32_t w = bl.upd[d.upd_off + b2];
            if (w < 0 || w >= n) { ++bad; continue; }
            v[d.p + b2] = u[w];
            if (std::isnan(v[d.p + b2])) ++nanreads;
          }
          for (int row = it.row0; row < it.row0 + it.nrows; ++row) {
            double sum = 0;
            for (int j = row; j < f; ++j) sum += bl.B[d.boff + (int64_t)row * d.bld + j] * v[j];
            wu.push_back({d.pos0 + row, sum});
          }
        }
      }
    }
    for (auto& q : wy) y[q.first] = q.second;
    for (auto& q : wc) cb[q.first] = q.second;
    for (auto& q : wu) u[q.first] = q.second;
    for (auto& q : wrp) rp[q.first] = q.second;
  }
  for (size_t t = 0; t < bl.nodes.size(); ++t)
    if (bl.nodes[t].height >= kmin && (fcover[t] != bl.nodes[t].p + bl.nodes[t].u || bcover[t] != bl.nodes[t].p))
      ++bad;
  printf("block form, split %d: %zu items, largest front %d, bad %d, nan-reads %d\n", kmin, bl.items.size(),
         bl.max_front, bad, nanreads);
  return bad + nanreads;
}

void parse_shapes(int argc, char** argv, int a0, std::vector<int>& nb, std::vector<int>& wpb) {
  for (int a = a0; a < argc; ++a) {
    nb.push_back(atoi(argv[a]));
    const char* c = std::strchr(argv[a], ':');
    wpb.push_back(c ? atoi(c + 1) : 1);
  }
}

void make_problem(int dim, int ne, int nsub, int jitter, std::vector<double>& sig, std::vector<int32_t>& part) {
  const int64_t nel = dim == 3 ? (int64_t)ne * ne * ne : (int64_t)ne * ne;
  sig.resize(nel);
  part.resize(nel);
  std::mt19937 g(7);
  std::lognormal_distribution<double> ln(0, 1);
  std::uniform_int_distribution<int> ud(0, 2);
  const int H = ne / nsub;
  for (int64_t e = 0; e < nel; ++e) {
    sig[e] = ln(g);
    int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = dim == 3 ? (int)(e / ((int64_t)ne * ne)) : 0;
    if (jitter) ex = std::min(ne - 1, ex + ud(g));
    part[e] = ex / H + nsub * (ey / H + nsub * (ez / H));
  }
}

}  // namespace

static int coarse_mode(int argc, char** argv) {
  if (argc < 5) return 2;
  const int ne = atoi(argv[1]), nsub = atoi(argv[2]), jitter = atoi(argv[3]);
  std::vector<int> nb, wpb;
  parse_shapes(argc, argv, 4, nb, wpb);
  std::vector<double> sig;
  std::vector<int32_t> part;
  make_problem(3, ne, nsub, jitter, sig, part);
  bddc_problem_t P{3, ne, sig.data(), part.data(), nsub * nsub * nsub};
  bddc_options_t O{};
  O.nrhs_max = 1;
  O.coarse = BDDC_COARSE_SPARSE;
  HostSetup hs;
  std::string err;
  if (host_setup(&P, &O, hs, err, true, true) != BDDC_OK) {
    printf("setup failed: %s\n", err.c_str());
    return 1;
  }
  std::vector<int32_t> perm;
  coarse_renumber(hs.cfac, perm);
  const CoarseFactor& cf = hs.cfac;
  const int n = (int)cf.n;
  GatherLayout gl;
  gather_layout(cf, (int)nb.size(), nb.data(), wpb.data(), gl);
  std::vector<double> r0(n), r(n);
  for (int i = 0; i < n; ++i) r0[i] = std::sin(0.37 * i) + 0.1;
  for (int i = 0; i < n; ++i) r[perm[i]] = r0[i];   // device numbering
  int bad = 0;
  std::vector<std::vector<double>> us;
  for (size_t sh = 0; sh < nb.size(); ++sh) {
    std::vector<double> u;
    bad += emulate(cf, gl, (int)sh, nb[sh] * wpb[sh], r, u, "coarse");
    double en = 0, rn = 0;
    for (int i = 0; i < n; ++i) {
      double a = 0;
      for (int64_t j = hs.Ac_ptr[i]; j < hs.Ac_ptr[i + 1]; ++j) a += hs.Ac_val[j] * u[perm[hs.Ac_col[j]]];
      en += (a - r0[i]) * (a - r0[i]);
      rn += r0[i] * r0[i];
    }
    const double res = std::sqrt(en / rn);
    printf("  A_c u = r residual %.2e\n", res);
    if (!(res < 1e-12)) ++bad;
    us.push_back(u);
  }
  {
    // the per-level form of the same layout (one launch per phase)
    GatherLayout one = gl;
    one.units.assign(1, gl.seq);
    one.wo.assign(1, std::vector<int32_t>());
    for (size_t ph = 0; ph + 1 < gl.seq_off.size(); ++ph) {
      one.wo[0].push_back((int32_t)gl.seq_off[ph]);
      one.wo[0].push_back((int32_t)gl.seq_off[ph + 1]);
    }
    std::vector<double> u;
    bad += emulate(cf, one, 0, 1, r, u, "coarse per-level form");
    double en = 0, rn = 0;
    for (int i = 0; i < n; ++i) {
      double a = 0;
      for (int64_t j = hs.Ac_ptr[i]; j < hs.Ac_ptr[i + 1]; ++j) a += hs.Ac_val[j] * u[perm[hs.Ac_col[j]]];
      en += (a - r0[i]) * (a - r0[i]);
      rn += r0[i] * r0[i];
    }
    printf("  A_c u = r residual %.2e\n", std::sqrt(en / rn));
    if (!(std::sqrt(en / rn) < 1e-12)) ++bad;
  }
  for (size_t sh = 1; sh < us.size(); ++sh)
    for (int i = 0; i < n; ++i)
      if (us[sh][i] != us[0][i]) {
        ++bad;
        break;
      }
  printf("%s\n", bad ? "FAILED" : "ok");
  return bad ? 1 : 0;
}

static double rel_diff(const std::vector<double>& a, const std::vector<double>& b) {
  if (a.size() != b.size()) return 1e300;
  double d = 0, m = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    d = std::max(d, std::fabs(a[i] - b[i]));
    m = std::max(m, std::fabs(b[i]));
  }
  return m > 0 ? d / m : d;
}

static int local_mode(int argc, char** argv) {
  if (argc < 8) return 2;
  const int dim = atoi(argv[2]), ne = atoi(argv[3]), nsub = atoi(argv[4]), jitter = atoi(argv[5]),
            leaf = atoi(argv[6]);
  std::vector<int> nb, wpb;
  parse_shapes(argc, argv, 7, nb, wpb);
  std::vector<double> sig;
  std::vector<int32_t> part;
  make_problem(dim, ne, nsub, jitter, sig, part);
  const int S = dim == 3 ? nsub * nsub * nsub : nsub * nsub;
  bddc_problem_t P{dim, ne, sig.data(), part.data(), S};
  bddc_options_t O{};
  O.nrhs_max = 1;
  O.coarse = BDDC_COARSE_DENSE;
  HostSetup hd, hsp;
  std::string err;
  if (host_setup(&P, &O, hd, err, false, true) != BDDC_OK) {
    printf("dense setup failed: %s\n", err.c_str());
    return 1;
  }
  O.local_solver = BDDC_LOCAL_SPARSE;
  O.local_leaf = leaf;
  if (host_setup(&P, &O, hsp, err, false, true) != BDDC_OK) {
    printf("sparse setup failed: %s\n", err.c_str());
    return 1;
  }
  int bad = 0;
  double worst = 0;
  for (int s = 0; s < S; ++s) {
    if (hsp.agi_ptr[s] != hd.agi_ptr[s] || hsp.agi_col[s] != hd.agi_col[s] || hsp.agi_val[s] != hd.agi_val[s] ||
        hsp.aig_ptr[s] != hd.aig_ptr[s] || hsp.aig_col[s] != hd.aig_col[s] || hsp.aig_val[s] != hd.aig_val[s])
      ++bad;
    worst = std::max(worst, rel_diff(hsp.Kgg[s], hd.Kgg[s]));
    worst = std::max(worst, rel_diff(hsp.Phi[s], hd.Phi[s]));
    worst = std::max(worst, rel_diff(hsp.Aci[s], hd.Aci[s]));
    if (!hsp.AIIinv[s].empty() || (int64_t)hsp.ifac[s].n != (int64_t)hsp.sub_I[s].size()) ++bad;
  }
  printf("local: %d subdomains, couplings %s, K_GG / Phi_G / A_ci largest relative difference %.2e\n", S,
         bad ? "DIFFER" : "equal", worst);
  if (!(worst < 1e-10)) ++bad;
  // the forest, as the device builds it
  std::vector<int32_t> ioff(S + 1, 0);
  std::vector<std::vector<int32_t>> iperm(S);
  int lmax = 0;
  for (int s = 0; s < S; ++s) {
    ioff[s + 1] = ioff[s] + (int32_t)hsp.sub_I[s].size();
    coarse_renumber(hsp.ifac[s], iperm[s]);
    lmax = std::max(lmax, hsp.ifac[s].n_levels);
  }
  CoarseFactor forest;
  merge_forest(hsp.ifac, ioff, forest);
  if (forest.n != ioff[S] || forest.n_levels != lmax) ++bad;
  for (int64_t i = 0; i < forest.n; ++i)
    if (forest.order[i] != i) ++bad;
  const int n = (int)forest.n;
  GatherLayout gl;
  gather_layout(forest, (int)nb.size(), nb.data(), wpb.data(), gl);
  std::vector<double> r(n);
  for (int i = 0; i < n; ++i) r[i] = std::sin(0.61 * i) + 0.2 * std::cos(1.3 * i);
  std::vector<std::vector<double>> us;
  for (size_t sh = 0; sh < nb.size(); ++sh) {
    std::vector<double> u;
    bad += emulate(forest, gl, (int)sh, nb[sh] * wpb[sh], r, u, "interior forest");
    double err2 = 0;
    for (int s = 0; s < S; ++s) {
      const int nI = ioff[s + 1] - ioff[s];
      std::vector<double> xd(nI, 0.0), xs(nI);
      for (int l = 0; l < nI; ++l) {
        for (int m = 0; m < nI; ++m) xd[l] += hd.AIIinv[s][(size_t)l * nI + m] * r[ioff[s] + iperm[s][m]];
        xs[l] = u[ioff[s] + iperm[s][l]];
      }
      err2 = std::max(err2, rel_diff(xs, xd));
    }
    printf("  sweeps against the dense A_II^-1 r: largest relative difference %.2e\n", err2);
    if (!(err2 < 1e-10)) ++bad;
    us.push_back(u);
  }
  // the per-level form: class ranges and block counts of every phase, and
  // the sweeps with each phase's units in storage order (one launch per
  // phase) give bitwise the result of the shapes above
  {
    std::vector<SweepSet::LevelPhase> lv;
    level_phases(gl, lv);
    int lbad = 0;
    if ((int)lv.size() != 2 * forest.n_levels || gl.seq_off.back() != (int64_t)gl.seq.size()) ++lbad;
    for (size_t ph = 0; ph < lv.size(); ++ph) {
      const SweepSet::LevelPhase& P = lv[ph];
      const int64_t m = gl.seq_off[ph + 1] - gl.seq_off[ph];
      if (P.u0 != gl.seq_off[ph] || P.cb[0] != 0 || P.cb[kLevelClasses] != m || P.bb[0] != 0) ++lbad;
      for (int c = 0; c < kLevelClasses; ++c) {
        const int per = kLevelThreads / kLevelGroup[c];
        const int cnt = P.cb[c + 1] - P.cb[c];
        if (cnt < 0 || P.bb[c + 1] - P.bb[c] != (cnt + per - 1) / per) ++lbad;
        for (int k = P.cb[c]; k < P.cb[c + 1]; ++k)
          if (level_class(gl.seq[P.u0 + k].len) != c) ++lbad;
      }
    }
    GatherLayout one = gl;
    one.units.assign(1, gl.seq);
    one.wo.assign(1, std::vector<int32_t>());
    for (size_t ph = 0; ph < lv.size(); ++ph) {
      one.wo[0].push_back((int32_t)gl.seq_off[ph]);
      one.wo[0].push_back((int32_t)gl.seq_off[ph + 1]);
    }
    std::vector<double> u;
    lbad += emulate(forest, one, 0, 1, r, u, "per-level form");
    for (int i = 0; i < n && !us.empty(); ++i)
      if (u[i] != us[0][i]) {
        ++lbad;
        break;
      }
    printf("  per-level form: %zu phases, %s\n", lv.size(), lbad ? "FAILED" : "ok");
    bad += lbad;
  }
  // the block form, with chunks small enough that big nodes span several,
  // pure and split at every height
  GatherLayout gseq;
  gather_layout(forest, 0, nullptr, nullptr, gseq);
  for (int64_t target : {64, 4096})
  for (int kmin = 0; kmin <= forest.n_levels; kmin += (target == 64 ? 1 : forest.n_levels)) {
    BlockLayout bl;
    block_layout(forest, target, bl);
    std::vector<double> u;
    int bbad = emulate_block(forest, bl, gseq, kmin, r, u);
    double err2 = 0;
    for (int s = 0; s < S; ++s) {
      const int nI = ioff[s + 1] - ioff[s];
      std::vector<double> xd(nI, 0.0), xs(nI);
      for (int l = 0; l < nI; ++l) {
        for (int m = 0; m < nI; ++m) xd[l] += hd.AIIinv[s][(size_t)l * nI + m] * r[ioff[s] + iperm[s][m]];
        xs[l] = u[ioff[s] + iperm[s][l]];
      }
      err2 = std::max(err2, rel_diff(xs, xd));
    }
    printf("  block form (chunks of %lld entries, split %d) against the dense A_II^-1 r: %.2e\n", (long long)target,
           kmin, err2);
    if (!(err2 < 1e-10)) ++bbad;
    bad += bbad;
  }
  for (size_t sh = 1; sh < us.size(); ++sh)
    for (int i = 0; i < n; ++i)
      if (us[sh][i] != us[0][i]) {
        ++bad;
        break;
      }
  printf("levels %d, entries %lld\n", forest.n_levels, (long long)forest.nnz);
  printf("%s\n", bad ? "FAILED" : "ok");
  return bad ? 1 : 0;
}

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "local") == 0) return local_mode(argc, argv);
  return coarse_mode(argc, argv);
}
