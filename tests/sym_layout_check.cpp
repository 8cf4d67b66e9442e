// Host check of the lower-triangle layout of the symmetric streamed GEMV
// (test helper, built and run by test_sym_layout_host.py): for every
// operator size n <= 128 V and a range of stage sizes, the closed-form
// offsets equal the sums of the padded row lengths, and the closed-form
// stage end equals the largest block-row count that fits (linear search),
// so the stages tile [0, n) with whole block-rows of at most stage_elems.
#include <cstdio>
#include <cstdlib>

#include "../paper_2410_14786_gb300/csrc/sym_layout.hpp"

using namespace bddc;

template <int V>
long check(int se_step) {
  long bad = 0, cases = 0;
  for (int n = 1; n <= 128 * V; ++n) {
    // offsets: row g holds g + 1 entries padded to a multiple of V
    long long sum = 0;
    for (int g = 0; g <= n; ++g) {
      if (tri_off<V>(g) != sum) ++bad;
      sum += (long long)V * (g / V + 1);
    }
    const int nblk = (n + V - 1) / V;
    for (int G = 0; G <= nblk; ++G)
      if (blk_off<V>(G, n) != tri_off<V>(V * G < n ? V * G : n)) ++bad;
    // stages: the widest block-row is the smallest stage
    const int minst = nblk * V * V;
    for (int se = minst; se <= 60000; se += (se < minst + 2048 ? 1 : se_step)) {
      for (int G0 = 0; G0 < nblk;) {
        ++cases;
        const int32_t base = blk_off<V>(G0, n);
        int lin = G0 + 1;
        while (lin < nblk && blk_off<V>(lin + 1, n) - base <= se) ++lin;
        const int G1 = sym_stage_end<V>(G0, nblk, n, se);
        if (G1 != lin || G1 <= G0 || G1 > nblk || blk_off<V>(G1, n) - base > se) {
          if (bad < 5) printf("V=%d n=%d se=%d G0=%d: closed %d linear %d\n", V, n, se, G0, G1, lin);
          ++bad;
          break;
        }
        G0 = G1;
      }
    }
  }
  printf("V=%d: %ld stage cases, %ld mismatches\n", V, cases, bad);
  return bad;
}

int main(int argc, char** argv) {
  const int step = argc > 1 ? atoi(argv[1]) : 97;
  const long bad = check<8>(step) + check<4>(step);
  printf(bad ? "FAILED\n" : "ok\n");
  return bad ? 1 : 0;
}
