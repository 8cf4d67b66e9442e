// Dense float64 linear algebra for the host-side setup (row-major storage).
//
// Setup needs, per subdomain and once for the coarse matrix: Cholesky
// factorisations, explicit inverses of SPD matrices and matrix products.
// These are plain blocked algorithms: a packed GEMM with a 4x8 register
// block, a right-looking blocked Cholesky, a column-block-parallel
// triangular inverse and the product L^-T L^-1. All loops keep the
// contiguous index innermost so that the compiler vectorises them without
// reassociating sums; no architecture-specific code.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace bddc {

// Run f(t) for t in [0, n) on up to `threads` std::threads (dynamic split).
template <typename F>
inline void parallel_for(int64_t n, int threads, F&& f) {
  if (n <= 0) return;
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, n));
  if (threads == 1) {
    for (int64_t t = 0; t < n; ++t) f(t);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> pool;
  pool.reserve(threads);
  for (int w = 0; w < threads; ++w)
    pool.emplace_back([&]() {
      for (int64_t t; (t = next.fetch_add(1)) < n;) f(t);
    });
  for (auto& th : pool) th.join();
}

namespace dense {

constexpr int MR = 4, NR = 8;        // register block
constexpr int MC = 128, KC = 256, NC = 2048;

// C[m x n] += alpha * op(A)[m x k] * op(B)[k x n].
// op(A) = A (row-major, lda) or A^T when ta; op(B) likewise with tb.
struct GemmArgs {
  int m, n, k;
  double alpha;
  const double* A; int64_t lda; bool ta;
  const double* B; int64_t ldb; bool tb;
  double* C; int64_t ldc;
};

inline double opA(const GemmArgs& g, int64_t i, int64_t p) {
  return g.ta ? g.A[p * g.lda + i] : g.A[i * g.lda + p];
}
inline double opB(const GemmArgs& g, int64_t p, int64_t j) {
  return g.tb ? g.B[j * g.ldb + p] : g.B[p * g.ldb + j];
}

// Pack op(A)[i0:i0+mc, p0:p0+kc] as MR-row slivers: Ap[s][p][r].
inline void pack_a(const GemmArgs& g, int i0, int mc, int p0, int kc, double* Ap) {
  for (int s = 0; s < mc; s += MR) {
    double* dst = Ap + (int64_t)s * kc;
    int rows = std::min(MR, mc - s);
    if (!g.ta) {
      for (int r = 0; r < MR; ++r) {
        if (r < rows) {
          const double* src = g.A + (int64_t)(i0 + s + r) * g.lda + p0;
          for (int p = 0; p < kc; ++p) dst[p * MR + r] = src[p];
        } else {
          for (int p = 0; p < kc; ++p) dst[p * MR + r] = 0.0;
        }
      }
    } else {
      for (int p = 0; p < kc; ++p) {
        const double* src = g.A + (int64_t)(p0 + p) * g.lda + i0 + s;
        for (int r = 0; r < MR; ++r) dst[p * MR + r] = r < rows ? src[r] : 0.0;
      }
    }
  }
}

// Pack op(B)[p0:p0+kc, j0:j0+nc] as NR-column slivers: Bp[s][p][c].
inline void pack_b(const GemmArgs& g, int p0, int kc, int j0, int nc, double* Bp) {
  for (int s = 0; s < nc; s += NR) {
    double* dst = Bp + (int64_t)s * kc;
    int cols = std::min(NR, nc - s);
    if (!g.tb) {
      for (int p = 0; p < kc; ++p) {
        const double* src = g.B + (int64_t)(p0 + p) * g.ldb + j0 + s;
        for (int c = 0; c < NR; ++c) dst[p * NR + c] = c < cols ? src[c] : 0.0;
      }
    } else {
      for (int c = 0; c < NR; ++c) {
        if (c < cols) {
          const double* src = g.B + (int64_t)(j0 + s + c) * g.ldb + p0;
          for (int p = 0; p < kc; ++p) dst[p * NR + c] = src[p];
        } else {
          for (int p = 0; p < kc; ++p) dst[p * NR + c] = 0.0;
        }
      }
    }
  }
}

inline void micro(int kc, const double* __restrict a, const double* __restrict b, double alpha,
                  double* __restrict C, int64_t ldc, int rows, int cols) {
  double acc[MR][NR];
  for (int r = 0; r < MR; ++r)
    for (int c = 0; c < NR; ++c) acc[r][c] = 0.0;
  for (int p = 0; p < kc; ++p) {
    const double* bp = b + p * NR;
    const double* ap = a + p * MR;
    for (int r = 0; r < MR; ++r) {
      const double av = ap[r];
      for (int c = 0; c < NR; ++c) acc[r][c] += av * bp[c];
    }
  }
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) C[r * ldc + c] += alpha * acc[r][c];
}

// Single-threaded GEMM over the row range [i_begin, i_end) of C.
inline void gemm_rows(const GemmArgs& g, int i_begin, int i_end, std::vector<double>& Ap,
                      std::vector<double>& Bp) {
  Ap.resize((size_t)MC * KC);
  Bp.resize((size_t)KC * NC);
  for (int j0 = 0; j0 < g.n; j0 += NC) {
    int nc = std::min(NC, g.n - j0);
    for (int p0 = 0; p0 < g.k; p0 += KC) {
      int kc = std::min(KC, g.k - p0);
      pack_b(g, p0, kc, j0, nc, Bp.data());
      for (int i0 = i_begin; i0 < i_end; i0 += MC) {
        int mc = std::min(MC, i_end - i0);
        pack_a(g, i0, mc, p0, kc, Ap.data());
        for (int js = 0; js < nc; js += NR)
          for (int is = 0; is < mc; is += MR)
            micro(kc, Ap.data() + (int64_t)is * kc, Bp.data() + (int64_t)js * kc, g.alpha,
                  g.C + (int64_t)(i0 + is) * g.ldc + j0 + js, g.ldc, std::min(MR, mc - is),
                  std::min(NR, nc - js));
      }
    }
  }
}

inline void gemm(const GemmArgs& g, int threads = 1) {
  if (g.m <= 0 || g.n <= 0 || g.k <= 0) return;
  int nblk = (g.m + MC - 1) / MC;
  if (threads <= 1 || nblk == 1) {
    std::vector<double> Ap, Bp;
    gemm_rows(g, 0, g.m, Ap, Bp);
    return;
  }
  parallel_for(nblk, threads, [&](int64_t b) {
    thread_local std::vector<double> Ap, Bp;
    int i0 = (int)b * MC;
    gemm_rows(g, i0, std::min(g.m, i0 + MC), Ap, Bp);
  });
}

// C += alpha * A * B (no transposes) convenience wrapper.
inline void gemm_nn(int m, int n, int k, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double* C, int64_t ldc, int threads = 1) {
  gemm(GemmArgs{m, n, k, alpha, A, lda, false, B, ldb, false, C, ldc}, threads);
}

// Unblocked lower Cholesky of the n x n block at A (row-major, lda); the
// lower triangle becomes L. Returns -1, or the index of the first pivot
// that is not above `min_pivot` (singular or indefinite to working accuracy).
inline int potrf_unblocked(int n, double* A, int64_t lda, double min_pivot = 0.0) {
  for (int j = 0; j < n; ++j) {
    double* Aj = A + (int64_t)j * lda;
    double d = Aj[j];
    for (int k = 0; k < j; ++k) d -= Aj[k] * Aj[k];
    if (!(d > min_pivot) || !std::isfinite(d)) return j;
    d = std::sqrt(d);
    Aj[j] = d;
    const double inv = 1.0 / d;
    for (int i = j + 1; i < n; ++i) {
      double* Ai = A + (int64_t)i * lda;
      double s = Ai[j];
      for (int k = 0; k < j; ++k) s -= Ai[k] * Aj[k];
      Ai[j] = s * inv;
    }
  }
  return -1;
}

// Blocked right-looking lower Cholesky; the strict upper triangle is zeroed.
// A pivot not above 1e-12 times the largest diagonal entry counts as a
// failure: the matrix is singular to working accuracy (e.g. the Schur
// complement of a floating subdomain without constraints).
inline int potrf(int n, double* A, int64_t lda, int threads = 1) {
  const int nb = 96;
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = std::max(dmax, std::fabs(A[(int64_t)i * lda + i]));
  const double min_pivot = 1e-12 * dmax;
  for (int k0 = 0; k0 < n; k0 += nb) {
    int b = std::min(nb, n - k0);
    double* Akk = A + (int64_t)k0 * lda + k0;
    int bad = potrf_unblocked(b, Akk, lda, min_pivot);
    if (bad >= 0) return k0 + bad;
    int m = n - k0 - b;
    if (m == 0) break;
    // panel: L21 = A21 * L11^-T, row by row (forward substitution)
    double* A21 = A + (int64_t)(k0 + b) * lda + k0;
    parallel_for(m, threads > 1 && m > 256 ? threads : 1, [&](int64_t i) {
      double* row = A21 + i * lda;
      for (int j = 0; j < b; ++j) {
        const double* Lj = Akk + (int64_t)j * lda;
        double s = row[j];
        for (int q = 0; q < j; ++q) s -= row[q] * Lj[q];
        row[j] = s / Lj[j];
      }
    });
    // trailing update, lower block triangle only: A22 -= L21 L21^T
    const int tb = MC;
    int nblk = (m + tb - 1) / tb;
    int64_t npairs = (int64_t)nblk * (nblk + 1) / 2;
    parallel_for(npairs, threads, [&](int64_t t) {
      int I = 0;
      while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
      int J = (int)(t - (int64_t)I * (I + 1) / 2);
      int i0 = I * tb, j0 = J * tb;
      int mi = std::min(tb, m - i0), nj = std::min(tb, m - j0);
      double* C = A + (int64_t)(k0 + b + i0) * lda + (k0 + b + j0);
      GemmArgs g{mi, nj, b, -1.0, A21 + (int64_t)i0 * lda, lda, false,
                 A21 + (int64_t)j0 * lda, lda, true, C, lda};
      std::vector<double> Ap, Bp;
      gemm_rows(g, 0, mi, Ap, Bp);
    });
  }
  for (int i = 0; i < n; ++i)
    std::fill(A + (int64_t)i * lda + i + 1, A + (int64_t)i * lda + n, 0.0);
  return -1;
}

// X = L^-1 for lower-triangular L (n x n, lda); X is lower triangular.
// Block column J of X depends only on L, so block columns run in parallel.
inline void trtri_lower(int n, const double* L, int64_t lda, double* X, int64_t ldx,
                        int threads = 1) {
  const int nb = 64;
  int nblk = (n + nb - 1) / nb;
  for (int i = 0; i < n; ++i) std::fill(X + (int64_t)i * ldx, X + (int64_t)i * ldx + n, 0.0);
  // inverse of each diagonal block (unblocked, column by column)
  parallel_for(nblk, threads, [&](int64_t B) {
    int o = (int)B * nb, b = std::min(nb, n - o);
    for (int j = 0; j < b; ++j) {
      X[(int64_t)(o + j) * ldx + o + j] = 1.0 / L[(int64_t)(o + j) * lda + o + j];
      for (int i = j + 1; i < b; ++i) {
        double s = 0.0;
        for (int q = j; q < i; ++q) s += L[(int64_t)(o + i) * lda + o + q] * X[(int64_t)(o + q) * ldx + o + j];
        X[(int64_t)(o + i) * ldx + o + j] = -s / L[(int64_t)(o + i) * lda + o + i];
      }
    }
  });
  // off-diagonal blocks: X[I,J] = -X[I,I] * sum_{J<=K<I} L[I,K] X[K,J]
  parallel_for(nblk, threads, [&](int64_t Jb) {
    int J = (int)(nblk - 1 - Jb);        // biggest columns first
    int oj = J * nb, bj = std::min(nb, n - oj);
    std::vector<double> T((size_t)nb * nb), Ap, Bp;
    for (int I = J + 1; I < nblk; ++I) {
      int oi = I * nb, bi = std::min(nb, n - oi);
      std::fill(T.begin(), T.end(), 0.0);
      int kk = oi - oj;   // K spans columns [oj, oi)
      GemmArgs g{bi, bj, kk, 1.0, L + (int64_t)oi * lda + oj, lda, false,
                 X + (int64_t)oj * ldx + oj, ldx, false, T.data(), nb};
      gemm_rows(g, 0, bi, Ap, Bp);
      GemmArgs g2{bi, bj, bi, -1.0, X + (int64_t)oi * ldx + oi, ldx, false, T.data(), nb, false,
                  X + (int64_t)oi * ldx + oj, ldx};
      gemm_rows(g2, 0, bi, Ap, Bp);
    }
  });
}

// Ainv = X^T X with X = L^-1 lower triangular: the inverse of L L^T.
// Full symmetric result in Ainv (n x n, ld).
inline void lower_gram(int n, const double* X, int64_t ldx, double* Ainv, int64_t ld,
                       int threads = 1) {
  const int tb = MC;
  int nblk = (n + tb - 1) / tb;
  int64_t npairs = (int64_t)nblk * (nblk + 1) / 2;
  parallel_for(npairs, threads, [&](int64_t t) {
    int I = 0;
    while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
    int J = (int)(t - (int64_t)I * (I + 1) / 2);   // J <= I
    int oi = I * tb, oj = J * tb;
    int bi = std::min(tb, n - oi), bj = std::min(tb, n - oj);
    double* C = Ainv + (int64_t)oi * ld + oj;
    for (int r = 0; r < bi; ++r) std::fill(C + (int64_t)r * ld, C + (int64_t)r * ld + bj, 0.0);
    // (X^T X)[I,J] = sum over rows k >= oi of X[k, I]^T X[k, J]
    int k0 = oi;
    GemmArgs g{bi, bj, n - k0, 1.0, X + (int64_t)k0 * ldx + oi, ldx, true,
               X + (int64_t)k0 * ldx + oj, ldx, false, C, ld};
    std::vector<double> Ap, Bp;
    gemm_rows(g, 0, bi, Ap, Bp);
  });
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) Ainv[(int64_t)i * ld + j] = Ainv[(int64_t)j * ld + i];
}

// In-place inverse of an SPD matrix (n x n, lda) through its Cholesky
// factor. Returns -1 or the index of a non-positive pivot.
inline int spd_inverse(int n, double* A, int64_t lda, int threads = 1) {
  if (n == 0) return -1;
  int bad = potrf(n, A, lda, threads);
  if (bad >= 0) return bad;
  std::vector<double> X((size_t)n * n);
  trtri_lower(n, A, lda, X.data(), n, threads);
  lower_gram(n, X.data(), n, A, lda, threads);
  return -1;
}

}  // namespace dense
}  // namespace bddc
