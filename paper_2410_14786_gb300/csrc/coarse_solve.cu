// Coarse solve u_c = A_c^-1 r_c on the GPU from the supernodal factorisation
// of coarse_sparse.cpp (float64 throughout).
//
// Forward sweep, supernodes by increasing height (leaves first): for node t,
//   [y_P; c_t] = [L_PP^-1 ; M] r'_P,
// where r' starts as r_c and, after each level, every coarse dof that
// receives contributions from that level's nodes subtracts their sum
// (gathered through fixed lists, so the summation order never changes and
// results are reproducible). Backward sweep, by decreasing height:
//   u_P = [L_PP^-T , -M^T] [y_P ; u_U].
//
// The whole solve is one persistent cooperative kernel: blocks take the row
// tiles of a level round robin, then meet at a grid-wide barrier before the
// next phase. A barrier wait is bounded; on timeout the block records
// BDDC_ERR_TIMEOUT in the error flag and every block leaves at its next
// barrier. Values written by other blocks are read through L2 (__ldcg).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.hpp"
#include "kernels.cuh"

namespace bddc {

namespace {

constexpr int kThreads = 256;
constexpr int kRowTile = 16;
constexpr long long kBarrierCycles = 4000000000LL;   // about 2 s at 2 GHz

struct CoarseArgs {
  const CItem* items_f;
  const CItem* items_b;
  const CNodeDev* nodes;
  const double* F;
  const double* B;
  const int32_t* piv;
  const int32_t* upd;
  const int32_t* lvl;        // [L+1 forward item offsets][L+1 backward][L+1 receive][n_c]
  const int32_t* recv_dof;
  const int32_t* recv_ptr;   // per receive entry, its range of recv_slot
  const int32_t* recv_slot;
  const double* r;           // r_c
  double* rp;                // r'
  double* y;
  double* c;
  double* u;                 // u_c
  unsigned int* bar;         // [0] arrivals, [1] generation
  int32_t* err;
  int levels, nrhs, nb;
};

// Grid-wide barrier; false when a wait ran out (here or in another block).
__device__ bool grid_barrier(const CoarseArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* gen = a.bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(a.bar, 1u);
    if (arrived == gridDim.x - 1) {
      a.bar[0] = 0;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*(volatile int32_t*)a.err == BDDC_ERR_TIMEOUT || clock64() - t0 > kBarrierCycles) {
          atomicExch(a.err, BDDC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int32_t*)a.err == BDDC_ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// One row tile of a supernode matrix: stage the operand, one row per warp.
template <bool FWD>
__device__ void row_tile(const CoarseArgs& a, const CItem& it, double* xs) {
  const CNodeDev nd = a.nodes[it.node];
  const double* mat = FWD ? a.F : a.B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrhs = a.nrhs, nb = a.nb;
  for (int k0 = 0; k0 < nrhs; k0 += nb) {
    const int kn = min(nb, nrhs - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < it.ld * nb; i += kThreads) {
      const int j = i / nb, k = i - j * nb;
      double v = 0.0;
      if (k < kn && j < it.ncols) {
        const int col = k0 + k;
        if (FWD) {
          v = __ldcg(&a.rp[(int64_t)a.piv[nd.piv_off + j] * nrhs + col]);
        } else {
          v = j < nd.p ? __ldcg(&a.y[(int64_t)a.piv[nd.piv_off + j] * nrhs + col])
                       : __ldcg(&a.u[(int64_t)a.upd[nd.upd_off + j - nd.p] * nrhs + col]);
        }
      }
      xs[i] = v;
    }
    __syncthreads();
    for (int rr = warp; rr < it.nrows; rr += kThreads / 32) {
      const int row = it.row0 + rr;
      const double* m = mat + it.moff + (int64_t)row * it.ld;
      double acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = 0.0;
      for (int c0 = lane * 2; c0 < it.ld; c0 += 64) {
        const double2 mv = __ldg(reinterpret_cast<const double2*>(m + c0));
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k < kn) acc[k] = fma(mv.x, xs[c0 * nb + k], fma(mv.y, xs[(c0 + 1) * nb + k], acc[k]));
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
      double out = acc[0];
#pragma unroll
      for (int k = 1; k < 8; ++k)
        if (lane == k) out = acc[k];
      if (lane < kn) {
        const int col = k0 + lane;
        if (FWD) {
          if (row < nd.p) a.y[(int64_t)a.piv[nd.piv_off + row] * nrhs + col] = out;
          else a.c[(int64_t)(nd.c_off + row - nd.p) * nrhs + col] = out;
        } else {
          a.u[(int64_t)a.piv[nd.piv_off + row] * nrhs + col] = out;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_coarse_solve(CoarseArgs a) {
  extern __shared__ double xs[];
  const int L = a.levels;
  const int32_t* off_f = a.lvl;
  const int32_t* off_b = a.lvl + (L + 1);
  const int32_t* off_r = a.lvl + 2 * (L + 1);
  const int64_t n_c = a.lvl[3 * (L + 1)];
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kThreads;
  for (int64_t i = tid; i < n_c * a.nrhs; i += nthreads) a.rp[i] = a.r[i];   // r' = r_c
  if (!grid_barrier(a)) return;
  for (int lv = 0; lv < L; ++lv) {
    for (int t = off_f[lv] + blockIdx.x; t < off_f[lv + 1]; t += gridDim.x) row_tile<true>(a, a.items_f[t], xs);
    if (!grid_barrier(a)) return;
    if (off_r[lv + 1] > off_r[lv]) {
      const int64_t ne = (int64_t)(off_r[lv + 1] - off_r[lv]) * a.nrhs;
      for (int64_t i = tid; i < ne; i += nthreads) {
        const int e = off_r[lv] + (int)(i / a.nrhs);
        const int k = (int)(i % a.nrhs);
        double s = 0.0;
        for (int q = a.recv_ptr[e]; q < a.recv_ptr[e + 1]; ++q) s += __ldcg(&a.c[(int64_t)a.recv_slot[q] * a.nrhs + k]);
        double* dst = &a.rp[(int64_t)a.recv_dof[e] * a.nrhs + k];
        *dst = __ldcg(dst) - s;
      }
      if (!grid_barrier(a)) return;
    }
  }
  for (int lv = L - 1; lv >= 0; --lv) {
    for (int t = off_b[lv] + blockIdx.x; t < off_b[lv + 1]; t += gridDim.x) row_tile<false>(a, a.items_b[t], xs);
    if (lv > 0 && !grid_barrier(a)) return;
  }
}

template <typename T>
cudaError_t up(bddc_handle_s* h, T** dst, const std::vector<T>& v) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocations.push_back(p);
  *dst = static_cast<T*>(p);
  if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

cudaError_t build_coarse_device(bddc_handle_s* h, const CoarseFactor& cf) {
  const int L = cf.n_levels;
  h->c_levels = L;
  if (cf.n == 0) return cudaSuccess;
  const int nn = (int)cf.nodes.size();
  std::vector<CNodeDev> nodes(nn);
  std::vector<int32_t> piv, upd;
  std::vector<int64_t> foff(nn), boff(nn);
  std::vector<int32_t> fld(nn), bld(nn);
  int64_t fcur = 0, bcur = 0, ccur = 0;
  for (int t = 0; t < nn; ++t) {
    const CoarseNode& T = cf.nodes[t];
    nodes[t] = CNodeDev{T.p, T.u, (int32_t)piv.size(), (int32_t)upd.size(), (int32_t)ccur};
    piv.insert(piv.end(), T.piv.begin(), T.piv.end());
    upd.insert(upd.end(), T.upd.begin(), T.upd.end());
    ccur += T.u;
    fld[t] = (T.p + 1) / 2 * 2;
    bld[t] = (T.p + T.u + 1) / 2 * 2;
    fcur = (fcur + 31) / 32 * 32;
    foff[t] = fcur;
    fcur += (int64_t)(T.p + T.u) * fld[t];
    bcur = (bcur + 31) / 32 * 32;
    boff[t] = bcur;
    bcur += (int64_t)T.p * bld[t];
  }
  std::vector<double> F((size_t)std::max<int64_t>(fcur, 1), 0.0), B((size_t)std::max<int64_t>(bcur, 1), 0.0);
  for (int t = 0; t < nn; ++t) {
    const CoarseNode& T = cf.nodes[t];
    const int f = T.p + T.u;
    for (int r = 0; r < f; ++r)
      std::memcpy(&F[foff[t] + (int64_t)r * fld[t]], &T.Fm[(size_t)r * T.p], sizeof(double) * T.p);
    for (int r = 0; r < T.p; ++r)
      std::memcpy(&B[boff[t] + (int64_t)r * bld[t]], &T.Bm[(size_t)r * f], sizeof(double) * f);
  }
  // level table, work items and receive lists (per level: the dofs that the
  // level's nodes contribute to, each with its contribution slots in node
  // order; nodes without pivots contribute nothing)
  std::vector<int32_t> lvl(3 * (L + 1) + 1, 0);
  std::vector<CItem> itf, itb;
  std::vector<int32_t> recv_dof, recv_ptr(1, 0), recv_slot;
  std::vector<std::vector<int32_t>> slots_of(cf.n);
  std::vector<int32_t> touched;
  for (int lv = 0; lv < L; ++lv) {
    lvl[lv] = (int)itf.size();
    lvl[(L + 1) + lv] = (int)itb.size();
    lvl[2 * (L + 1) + lv] = (int)recv_dof.size();
    touched.clear();
    for (int t = 0; t < nn; ++t) {
      const CoarseNode& T = cf.nodes[t];
      if (T.height != lv || T.p == 0) continue;
      for (int r0 = 0; r0 < T.p + T.u; r0 += kRowTile)
        itf.push_back(CItem{foff[t], t, fld[t], T.p, r0, std::min(kRowTile, T.p + T.u - r0), 0});
      for (int r0 = 0; r0 < T.p; r0 += kRowTile)
        itb.push_back(CItem{boff[t], t, bld[t], T.p + T.u, r0, std::min(kRowTile, T.p - r0), 0});
      h->c_max_ld_f = std::max(h->c_max_ld_f, fld[t]);
      h->c_max_ld_b = std::max(h->c_max_ld_b, bld[t]);
      for (int a = 0; a < T.u; ++a) {
        const int32_t w = T.upd[a];
        if (slots_of[w].empty()) touched.push_back(w);
        slots_of[w].push_back(nodes[t].c_off + a);
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int32_t w : touched) {
      recv_dof.push_back(w);
      recv_slot.insert(recv_slot.end(), slots_of[w].begin(), slots_of[w].end());
      recv_ptr.push_back((int32_t)recv_slot.size());
      slots_of[w].clear();
    }
  }
  lvl[L] = (int)itf.size();
  lvl[(L + 1) + L] = (int)itb.size();
  lvl[2 * (L + 1) + L] = (int)recv_dof.size();
  lvl[3 * (L + 1)] = (int32_t)cf.n;
  h->c_nnz = fcur + bcur;
  h->c_update_total = ccur;
  cudaError_t e;
  if ((e = up(h, &h->d_cF, F)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_cB, B)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_citems_f, itf)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_citems_b, itb)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_cnodes, nodes)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_cpiv, piv)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_cupd, upd)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_clvl, lvl)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_crecv_dof, recv_dof)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_crecv_ptr, recv_ptr)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_crecv_slot, recv_slot)) != cudaSuccess) return e;
  if ((e = up(h, &h->d_cbar, std::vector<unsigned int>(2, 0u))) != cudaSuccess) return e;
  // cooperative grid: all blocks resident at once
  int dev = 0, sms = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  const int max_ld = std::max(h->c_max_ld_f, h->c_max_ld_b);
  int per_sm = 0;
  const size_t smem = (size_t)max_ld * 8 * sizeof(double);   // room for 8 right-hand sides
  if (smem > 48 * 1024 && (e = cudaFuncSetAttribute(k_coarse_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)std::min<size_t>(smem, 200 * 1024))) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_solve, kThreads,
                                                         std::min<size_t>(smem, 200 * 1024))) != cudaSuccess)
    return e;
  h->c_grid = sms * std::max(1, std::min(per_sm, 2));
  return cudaSuccess;
}

cudaError_t launch_coarse_solve(bddc_handle_s* h, const double* rc, double* uc, int nrhs, cudaStream_t st) {
  if (h->n_c == 0) return cudaSuccess;
  const int max_ld = std::max(h->c_max_ld_f, h->c_max_ld_b);
  int nb = std::min(nrhs, 8);
  while (nb > 1 && (size_t)max_ld * nb * sizeof(double) > 200 * 1024) nb >>= 1;
  const size_t smem = (size_t)max_ld * nb * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  CoarseArgs a{h->d_citems_f, h->d_citems_b, h->d_cnodes, h->d_cF, h->d_cB, h->d_cpiv, h->d_cupd, h->d_clvl,
               h->d_crecv_dof, h->d_crecv_ptr, h->d_crecv_slot, rc, h->w_cr, h->w_cy, h->w_cc, uc, h->d_cbar,
               h->d_err, h->c_levels, nrhs, nb};
  cudaError_t e = cudaMemsetAsync(h->d_cbar, 0, 2 * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->c_grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_coarse_solve, a);
  h->launches++;
  return e;
}

}  // namespace bddc
