// Host check of the gather form of the coarse sweeps (test helper, built and
// run by test_coarse_layout_host.py): sets up a 3D problem through the
// library's host setup, renumbers the coarse factor by elimination order,
// builds the gather layout for the given launch shapes, and emulates the
// sweeps phase by phase, warp by warp, unit by unit, as the kernel reads and
// writes them. Checks: every descriptor and index in range; within a phase
// no value read that the phase writes (except a receiving dof's own value);
// every position's y and u written exactly once; the result solves
// A_c u = r to 1e-12; and all shapes give bitwise the same u.
// Usage: coarse_layout_check ne nsub jitter blocks:wpb [blocks:wpb ...]
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

int main(int argc, char** argv) {
  if (argc < 5) return 2;
  const int ne = atoi(argv[1]), nsub = atoi(argv[2]), jitter = atoi(argv[3]);
  std::vector<int> nb, wpb;
  for (int a = 4; a < argc; ++a) {
    nb.push_back(atoi(argv[a]));
    const char* c = std::strchr(argv[a], ':');
    wpb.push_back(c ? atoi(c + 1) : 1);
  }
  const int64_t nel = (int64_t)ne * ne * ne;
  std::vector<double> sig(nel);
  std::vector<int32_t> part(nel);
  std::mt19937 g(7);
  std::lognormal_distribution<double> ln(0, 1);
  std::uniform_int_distribution<int> ud(0, 2);
  const int H = ne / nsub;
  for (int64_t e = 0; e < nel; ++e) {
    sig[e] = ln(g);
    int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = (int)(e / ((int64_t)ne * ne));
    if (jitter) ex = std::min(ne - 1, ex + ud(g));
    part[e] = ex / H + nsub * (ey / H + nsub * (ez / H));
  }
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
  const int n = (int)cf.n, L = cf.n_levels;
  GatherLayout gl;
  gather_layout(cf, (int)nb.size(), nb.data(), wpb.data(), gl);
  int bad = 0;
  for (int32_t ix : gl.I)
    if (ix < 0 || ix >= 2 * n) ++bad;
  std::vector<double> r0(n), r(n);
  for (int i = 0; i < n; ++i) r0[i] = std::sin(0.37 * i) + 0.1;
  for (int i = 0; i < n; ++i) r[perm[i]] = r0[i];   // device numbering
  std::vector<std::vector<double>> us;
  for (size_t sh = 0; sh < nb.size(); ++sh) {
    const int nw = nb[sh] * wpb[sh];
    const std::vector<CGUnit>& U = gl.units[sh];
    const std::vector<int32_t>& wo = gl.wo[sh];
    if (wo.size() != (size_t)2 * L * (nw + 1) || wo.front() != 0 || wo.back() != (int)U.size()) ++bad;
    for (size_t i = 1; i < wo.size(); ++i)
      if (wo[i] < wo[i - 1]) ++bad;
    for (const CGUnit& d : U)
      if (d.off < 0 || d.len < 1 || d.off + d.len > (int64_t)gl.C.size() || d.dst < 0 || d.dst >= n) ++bad;
    const double nan = std::nan("");
    std::vector<double> rp(n, nan), y(n, nan), u(n, nan);
    std::vector<int> ny(n, 0), nu(n, 0);
    int races = 0, nanreads = 0;
    for (int ph = 0; ph < 2 * L; ++ph) {
      const bool fwd = ph < L;
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
    double en = 0, rn = 0;
    for (int i = 0; i < n; ++i) {
      double a = 0;
      for (int64_t j = hs.Ac_ptr[i]; j < hs.Ac_ptr[i + 1]; ++j) a += hs.Ac_val[j] * u[perm[hs.Ac_col[j]]];
      en += (a - r0[i]) * (a - r0[i]);
      rn += r0[i] * r0[i];
    }
    const double res = std::sqrt(en / rn);
    printf("shape %d x %d: n_c %d levels %d races %d nan-reads %d write-count %d residual %.2e\n", nb[sh],
           wpb[sh], n, L, races, nanreads, once, res);
    if (races || nanreads || once || !(res < 1e-12)) ++bad;
    us.push_back(u);
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
