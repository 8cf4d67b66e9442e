// Layout of a symmetric operator stored as its lower triangle, read in
// block-rows (shared by the symmetric streamed GEMV and its host checks).
//
// Row g holds columns 0 .. g zero-padded to a multiple of V elements (16
// bytes), rows consecutive. Block-row G is rows V G .. V G + V - 1; all of
// them hold the same G + 1 vectors, so a block-row is contiguous and its
// offset has a closed form.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define SYM_HD __host__ __device__ __forceinline__
#else
#define SYM_HD inline
#endif

namespace bddc {

// Elements of rows 0 .. g - 1 of the stored triangle.
template <int V>
SYM_HD int64_t tri_off(int g) {
  const int64_t q = g / V, r = g % V;
  return (int64_t)V * (V * q * (q + 1) / 2 + r * (q + 1));
}

// Elements of block-rows 0 .. G - 1 of an n x n triangle (rows beyond n absent).
template <int V>
SYM_HD int32_t blk_off(int G, int n) {
  const int g = V * G < n ? V * G : n;
  const int q = g / V, r = g % V;
  return V * (V * q * (q + 1) / 2 + r * (q + 1));
}

// Block-rows [G0, G1) of one stage: as many whole block-rows as fit in
// stage_elems elements (at least one). Full block-rows (all but the
// operator's last) satisfy blk_off(G) = V^2 G (G + 1) / 2, so the largest G1
// solves a quadratic; the integer corrections make the float square root's
// rounding irrelevant, and the operator's last block-row, which may be
// partial, is checked with its exact size.
template <int V>
SYM_HD int sym_stage_end(int G0, int nblk, int n, int stage_elems) {
  const int C = G0 * (G0 + 1) + 2 * stage_elems / (V * V);
  int g = (int)((sqrtf(4.0f * (float)C + 1.0f) - 1.0f) * 0.5f);
  while ((g + 1) * (g + 2) <= C) ++g;
  while (g * (g + 1) > C) --g;
  if (g < G0 + 1) g = G0 + 1;
  if (g >= nblk) return nblk;
  if (g == nblk - 1 && blk_off<V>(nblk, n) - blk_off<V>(G0, n) <= stage_elems) return nblk;
  return g;
}

}  // namespace bddc
