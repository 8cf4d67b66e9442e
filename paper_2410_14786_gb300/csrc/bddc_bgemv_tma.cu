// Batched dense GEMV / skinny GEMM over many small operators, streamed from
// HBM with bulk asynchronous copies (cp.async.bulk, the TMA's 1D form) into
// a ring of shared-memory stages (sm_103a).
//
// Used for the local operators of the apply (A_II^-1 and K_GG of every
// subdomain): y = Op x with Op row-major, rows padded to 16 bytes. A work
// item is a run of consecutive rows of one operator, which is one contiguous
// byte range in the arena, so one bulk copy moves a whole stage of rows.
//
// Block layout: 8 consumer warps and 1 producer warp. The producer's lane 0
// walks the same (item, stage) sequence as the consumers and keeps up to
// kStages bulk copies in flight; `full[s]` completes when stage s has
// landed (transaction bytes), `empty[s]` when all 8 consumer warps are done
// with it. Consumers split each warp into groups of `lpr` lanes, one row per
// group, read the operator row from shared memory in 16-byte vectors, and
// reduce within the group. The operand x of the item is staged in shared
// memory (double buffered, one named barrier per item).
//
// Every mbarrier wait is bounded (kWaitCycles); on timeout the waiting
// thread sets *err and leaves its loop, and the producer waits (bounded) for
// its own copies in flight before the block exits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "kernels.cuh"
#include "sym_layout.hpp"

namespace bddc {

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kTmaThreads = (kConsumerWarps + 1) * 32;
constexpr int kStages = 4;
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// A waiting thread is suspended until the phase completes or kSuspendNs
// nanoseconds have passed, instead of polling.
constexpr uint32_t kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32) : "memory");
}

template <typename T> struct Op;
template <> struct Op<double> {
  static constexpr int V = 2;
  using Acc = double;
  __device__ static void load(const double* p, double o[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};
template <> struct Op<float> {
  static constexpr int V = 4;
  using Acc = float;
  __device__ static void load(const float* p, float o[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <> struct Op<__nv_bfloat16> {
  static constexpr int V = 8;
  using Acc = float;
  __device__ static void load(const __nv_bfloat16* p, float o[8]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};

// One 16-byte shared-memory load of accumulator-typed values.
__device__ __forceinline__ void load16(const float* p, float o[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load16(const double* p, double o[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x; o[1] = v.y;
}

// Register blocking for a block of NRB right-hand sides. With NRB >= 4 a
// group of kWideLanes lanes computes kRowsWide consecutive rows at once, so
// each x value read from shared memory feeds kRowsWide FMAs.
constexpr int kWideLanes = 16;
constexpr int kRowsWide = 4;
template <int NRB> struct Blocking {
  static constexpr bool wide = NRB >= 4;
  static constexpr int R = wide ? kRowsWide : 1;     // rows per lane group
};

// Lanes per row: for NRB >= 4 a fixed 16; otherwise the smallest power of
// two in [4, 32] that leaves each lane at most 8 vectors of the row, except
// that float64 operators (V = 2) allow up to 32 vectors per lane: that kernel is
// bound by GB300's float64 pipe, where a row's reduction (one DADD per
// halving) and its partly idle last step cost as much as its products, so
// fewer, fuller lanes per row do more useful work per instruction (8 lanes
// on a 343-column row: 91 % of the issued float64 lane operations are
// products, against 63 % with 32 lanes).
__host__ __device__ __forceinline__ int lanes_per_row(int lda, int V, int nrb) {
  if (nrb >= 4) return kWideLanes;
  const int nvec = (lda + V - 1) / V;
  const int cap = V == 2 ? 32 : 8;
  int l = 4;
  while (l < 32 && nvec > cap * l) l <<= 1;
  return l;
}
// Rows per stage: as many as fit, rounded down to whole warp groups (the
// rows one consumer warp computes in one pass: 32 / lpr groups of R rows).
__host__ __device__ __forceinline__ int rows_per_stage(int row_bytes, int stage_bytes, int wgr) {
  int rps = stage_bytes / row_bytes;
  if (rps >= wgr) rps = rps / wgr * wgr;
  return rps < 1 ? 1 : rps;
}

// Shared-memory layout of the operand x of one unit: columns in blocks of V
// (one 16-byte operator vector), each block holding its V x NRB values
// column-major by right-hand side, blocks padded to an odd number of 16-byte
// units. The lanes of a row group read consecutive blocks in the same
// instruction, and an odd stride puts the 8 lanes of each quarter warp on
// distinct banks.
template <typename Acc, int V, int NRB> struct XLayout {
  static constexpr int Q = 16 / (int)sizeof(Acc);   // values per 16-byte load
  static constexpr int U = V * NRB / Q;             // 16-byte loads per block
  static constexpr int XB = (U % 2 ? U : U + 1) * Q; // block stride (values)
  __host__ __device__ static constexpr size_t bytes(int lda) {
    return (size_t)((lda + V - 1) / V) * XB * sizeof(Acc);
  }
  __device__ static int index(int c, int k) { return (c / V) * XB + (c % V) * NRB + k; }
};

// Sum of the N accumulators of a row group over its L lanes, left
// distributed: after log2(L) halving exchanges, lane gl holds the sums of
// the flattened entries [gl * N / L, (gl + 1) * N / L) in v[0 .. N / L).
template <int N, int L, typename Acc>
__device__ __forceinline__ void reduce_scatter(Acc (&v)[N], int gl) {
  static_assert(N >= L && (L & (L - 1)) == 0, "reduce_scatter needs N >= L, L a power of two");
#pragma unroll
  for (int o = L / 2, n = N; o >= 1; o >>= 1, n >>= 1) {
    const bool upper = (gl & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const Acc send = upper ? v[i] : v[i + n / 2];
      const Acc keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

template <typename T, int NRB>
__global__ void __launch_bounds__(kTmaThreads) __maxnreg__(Blocking<NRB>::wide ? 112 : (NRB == 1 ? 56 : 72)) k_bgemv_tma(const WorkItem* __restrict__ items, int n_items,
                                                           const T* __restrict__ arena, const double* __restrict__ X,
                                                           double* __restrict__ Y,
                                                           const int32_t* __restrict__ yscatter, int nrhs,
                                                           int stage_bytes, int max_lda, int32_t* __restrict__ err) {
  using Acc = typename Op<T>::Acc;
  constexpr int V = Op<T>::V;
  using XL = XLayout<Acc, V, NRB>;
  constexpr int R = Blocking<NRB>::R;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stages = smem;
  Acc* xs = reinterpret_cast<Acc*>(smem + (size_t)kStages * stage_bytes);
  double* xraw = reinterpret_cast<double*>(smem + (size_t)kStages * stage_bytes + XL::bytes(max_lda));
  uint64_t* full = reinterpret_cast<uint64_t*>(xraw + (size_t)max_lda * NRB);
  uint64_t* empty = full + kStages;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int nrb = (nrhs + NRB - 1) / NRB;
  const int total = n_items * nrb;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    int slot = 0;
    uint32_t phase = 0;
    bool pending[kStages];
    uint32_t pend_parity[kStages];
    for (int s = 0; s < kStages; ++s) pending[s] = false;
    bool ok = true;
    for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const WorkItem w = items[u / nrb];
      const int row_bytes = w.lda * (int)sizeof(T);
      const int wgr = (32 / lanes_per_row(w.lda, V, NRB)) * R;
      const int rps = rows_per_stage(row_bytes, stage_bytes, wgr);
      for (int r0 = 0; r0 < w.nrows; r0 += rps) {
        if (!mbar_wait(&empty[slot], phase ^ 1u) || *(volatile int*)&abort_flag) {
          atomicExch(err, BDDC_ERR_TIMEOUT);
          abort_flag = 1;
          ok = false;
          break;
        }
        const int nr = min(rps, w.nrows - r0);
        const uint32_t bytes = (uint32_t)nr * (uint32_t)row_bytes;
        mbar_expect_tx(&full[slot], bytes);
        bulk_load(stages + (size_t)slot * stage_bytes, arena + w.moff + (int64_t)(w.row0 + r0) * w.lda, bytes,
                  &full[slot]);
        pending[slot] = true;
        pend_parity[slot] = phase;
        if (++slot == kStages) { slot = 0; phase ^= 1u; }
      }
    }
    // every copy this block issued must land before the block exits
    for (int s = 0; s < kStages; ++s)
      if (pending[s] && !mbar_wait(&full[s], pend_parity[s])) atomicExch(err, BDDC_ERR_TIMEOUT);
    return;
  }

  // ---------------- consumers ----------------
  // After a timeout a warp keeps walking the same units and reaches every
  // consumer barrier (so no other warp waits for it forever), but it no
  // longer waits on stages nor computes.
  // The fp64 operand of the next unit is copied into `xraw` with cp.async
  // while the current unit is computed, and converted into the padded
  // accumulator-typed layout `xs` when that unit starts, so staging the
  // operand costs no exposed global-memory latency.
  // The warp groups of a stage (wgr rows each) are dealt round-robin over the
  // consumer warps, continuing from the previous stage, so that every warp
  // has work even when a stage holds fewer rows than one pass of all warps.
  constexpr int kCT = kConsumerWarps * 32;
  const int tid = threadIdx.x;
  int slot = 0;
  uint32_t phase = 0;
  int turn = 0;   // consumer warp that takes the next warp group
  bool aborted = false;
  auto prefetch_operand = [&](int uu) {
    const WorkItem wn = items[uu / nrb];
    const int r0n = (uu % nrb) * NRB, nrn = min(NRB, nrhs - r0n);
    const int n = wn.lda * NRB;
    for (int i = tid; i < n; i += kCT) {
      const int c = i / NRB, k = i - c * NRB;
      if (c < wn.ncols && k < nrn)
        cp_async8(xraw + i, X + (int64_t)(wn.xoff + c) * nrhs + r0n + k);
      else
        xraw[i] = 0.0;
    }
    cp_async_commit();
  };
  if (blockIdx.x < total) prefetch_operand(blockIdx.x);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const WorkItem w = items[u / nrb];
    const int rhs0 = (u % nrb) * NRB;
    const int nr_rhs = min(NRB, nrhs - rhs0);
    const int nx = w.lda * NRB;
    cp_async_wait_all();
    consumer_sync();                          // operand of this unit landed; xs is free
    for (int i = tid; i < nx; i += kCT) {
      const int c = i / NRB, k = i - c * NRB;
      xs[XL::index(c, k)] = (Acc)xraw[i];
    }
    consumer_sync();                          // xs complete; xraw is free
    if (u + (int)gridDim.x < total) prefetch_operand(u + gridDim.x);
    const int lpr = lanes_per_row(w.lda, V, NRB);
    const int gpw = 32 / lpr;                 // lane groups per warp
    const int group = lane / lpr, gl = lane - group * lpr;
    const int wgr = gpw * R;                  // rows per warp group
    const int row_bytes = w.lda * (int)sizeof(T);
    const int rps = rows_per_stage(row_bytes, stage_bytes, wgr);
    for (int r0 = 0; r0 < w.nrows; r0 += rps) {
      if (!aborted && (*(volatile int*)&abort_flag || !mbar_wait(&full[slot], phase))) {
        if (lane == 0) atomicExch(err, BDDC_ERR_TIMEOUT);
        abort_flag = 1;
        aborted = true;
      }
      if (aborted) continue;
      const int nr = min(rps, w.nrows - r0);
      const int ngroups = (nr + wgr - 1) / wgr;
      const T* tile = reinterpret_cast<const T*>(stages + (size_t)slot * stage_bytes);
      int j = warp - turn;
      if (j < 0) j += kConsumerWarps;
      for (; j < ngroups; j += kConsumerWarps) {
        const int rb = j * wgr + group * R;     // first row of this lane group in the stage
        Acc acc[R * NRB];
#pragma unroll
        for (int e = 0; e < R * NRB; ++e) acc[e] = Acc(0);
        for (int c0 = gl * V; c0 < w.lda; c0 += lpr * V) {
          Acc av[R][V];
#pragma unroll
          for (int q = 0; q < R; ++q) {
            if (rb + q < nr) {
              Op<T>::load(tile + (size_t)(rb + q) * w.lda + c0, av[q]);
            } else {
#pragma unroll
              for (int v = 0; v < V; ++v) av[q][v] = Acc(0);
            }
          }
          const Acc* xb = xs + (c0 / V) * XL::XB;
#pragma unroll
          for (int uu = 0; uu < XL::U; ++uu) {
            Acc xq[XL::Q];
            load16(xb + uu * XL::Q, xq);
#pragma unroll
            for (int jj = 0; jj < XL::Q; ++jj) {
              const int e = uu * XL::Q + jj, v = e / NRB, k = e - v * NRB;
#pragma unroll
              for (int q = 0; q < R; ++q) acc[q * NRB + k] = fma(av[q][v], xq[jj], acc[q * NRB + k]);
            }
          }
        }
        const int64_t ybase = (int64_t)w.yoff + w.row0 + r0;
        if constexpr (Blocking<NRB>::wide) {
          constexpr int per = R * NRB / kWideLanes;
          reduce_scatter<R * NRB, kWideLanes>(acc, gl);
#pragma unroll
          for (int i = 0; i < per; ++i) {
            const int e = gl * per + i, q = e / NRB, k = e - q * NRB;
            if (rb + q < nr && k < nr_rhs) {
              const int64_t jy = ybase + rb + q;
              const int64_t dst = yscatter ? (int64_t)yscatter[jy] : jy;
              Y[dst * nrhs + rhs0 + k] = (double)acc[i];
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < NRB; ++k)
            for (int o = lpr >> 1; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
          // every lane of the group holds all NRB sums; lane gl writes the
          // columns k = gl, gl + lpr, ... (a group may have fewer lanes than NRB)
          if (rb < nr && gl < nr_rhs) {
            const int64_t jy = ybase + rb;
            const int64_t dst = yscatter ? (int64_t)yscatter[jy] : jy;
#pragma unroll
            for (int k = 0; k < NRB; ++k)
              if (k < nr_rhs && (k & (lpr - 1)) == gl) Y[dst * nrhs + rhs0 + k] = (double)acc[k];
          }
        }
      }
      turn = (turn + ngroups) % kConsumerWarps;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (++slot == kStages) { slot = 0; phase ^= 1u; }
    }
  }
  cp_async_wait_all();
}

// SM count of the current device, cached per device (every thread that
// fills an entry writes the same value).
constexpr int kMaxDevices = 64;
std::atomic<int> g_num_sms[kMaxDevices];
int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev >= kMaxDevices) {
    int n = 1;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return std::max(n, 1);
  }
  int n = g_num_sms[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    n = std::max(n, 1);
    g_num_sms[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// Shared memory of one block: kStages stages, two operand buffers, barriers.
template <typename T, int NRB>
size_t x_bytes(int max_lda) {
  return XLayout<typename Op<T>::Acc, Op<T>::V, NRB>::bytes(max_lda) + (size_t)max_lda * NRB * sizeof(double);
}
template <typename T, int NRB>
size_t block_smem(int stage_bytes, int max_lda) {
  return (size_t)kStages * stage_bytes + x_bytes<T, NRB>(max_lda) + 2 * kStages * sizeof(uint64_t);
}

// Stage size: about target_kb KB (12 by default; the autotuner may pick
// another) of rows of the widest operator (at least one row,
// a whole number of warp groups when that is possible), so that several
// blocks fit on an SM: measured on GB300 with 1728 bf16 operators of
// 343 x 344, four 12 KB stages per block and four blocks per SM streamed
// faster than fewer, larger stages.
template <typename T, int NRB>
int stage_size(int max_lda, int target_kb) {
  const long long row = (long long)max_lda * (long long)sizeof(T);
  const long long xs = (long long)x_bytes<T, NRB>(max_lda) + 2 * kStages * 8;
  const long long cap = (200LL * 1024 - xs) / kStages;
  const int wgr = (32 / lanes_per_row(max_lda, Op<T>::V, NRB)) * Blocking<NRB>::R;
  long long rows = std::max<long long>((long long)target_kb * 1024 / row, 1);
  if (rows >= wgr)
    rows = std::max<long long>((rows + wgr / 2) / wgr, 1) * wgr;
  else if ((long long)wgr * row <= cap)
    rows = wgr;   // wide rows: one whole warp group per stage rather than a partial one
  long long st = std::max<long long>(row, std::min<long long>(rows * row, cap));
  return (int)((st + 127) / 128 * 128);
}

template <typename T, int NRB>
cudaError_t run_tma(const WorkItem* items, int n_items, int max_lda, const T* arena, const double* X, double* Y,
                    const int32_t* yscatter, int nrhs, int32_t* err, cudaStream_t st, int stage_kb,
                    int max_per_sm) {
  const int stage_bytes = stage_size<T, NRB>(max_lda, stage_kb);
  const size_t smem = block_smem<T, NRB>(stage_bytes, max_lda);
  auto kern = k_bgemv_tma<T, NRB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaThreads, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, per_sm);
  if (max_per_sm > 0) per_sm = std::min(per_sm, max_per_sm);
  const int units = n_items * ((nrhs + NRB - 1) / NRB);
  const int grid = std::max(1, std::min(units, num_sms() * per_sm));
  kern<<<grid, kTmaThreads, smem, st>>>(items, n_items, arena, X, Y, yscatter, nrhs, stage_bytes, max_lda, err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const WorkItem* items, int n_items, int max_lda, const void* arena, const double* X, double* Y,
                     const int32_t* yscatter, int nrhs, int32_t* err, cudaStream_t st, int stage_kb,
                     int max_per_sm) {
  const T* A = static_cast<const T*>(arena);
  const size_t row = ((size_t)max_lda * sizeof(T) + 127) / 128 * 128;
  const size_t xb[4] = {x_bytes<T, 1>(max_lda), x_bytes<T, 2>(max_lda), x_bytes<T, 4>(max_lda),
                        x_bytes<T, 8>(max_lda)};
  auto fits = [&](int i) { return kStages * row + xb[i] + 64 <= 200 * 1024; };
  if (nrhs >= 8 && fits(3)) return run_tma<T, 8>(items, n_items, max_lda, A, X, Y, yscatter, nrhs, err, st,
                                                           stage_kb, max_per_sm);
  if (nrhs >= 4 && fits(2)) return run_tma<T, 4>(items, n_items, max_lda, A, X, Y, yscatter, nrhs, err, st,
                                                           stage_kb, max_per_sm);
  if (nrhs >= 2 && fits(1)) return run_tma<T, 2>(items, n_items, max_lda, A, X, Y, yscatter, nrhs, err, st,
                                                           stage_kb, max_per_sm);
  if (fits(0)) return run_tma<T, 1>(items, n_items, max_lda, A, X, Y, yscatter, nrhs, err, st,
                                                           stage_kb, max_per_sm);
  return cudaErrorInvalidValue;
}

// ---- symmetric operators: packed lower triangle -------------------------------------
//
// A symmetric operator A (n x n) is stored as L', its lower triangle with
// the diagonal halved, row g holding columns 0 .. g zero-padded to a multiple
// of V (16 bytes), rows consecutive: y = A x = L' x + L'^T x. Each stored
// entry a = L'[g, c] is read once and used twice, y[g] += a x[c] and
// yT[c] += a x[g] (the halved diagonal counts once in each), so the operator
// stream is about half of the full matrix.
//
// The kernel reads the triangle in block-rows: block-row G is rows V G ..
// V G + V - 1, every one of them holding the G + 1 vectors of columns 0 ..
// V G + V - 1, so a block-row is a V x (G + 1) array of V x V tiles,
// contiguous in the arena. One block owns one operator at a time (operators
// dealt round-robin over the blocks); its producer lane streams stages of
// whole block-rows with bulk copies (as in k_bgemv_tma) and publishes each
// stage's last block-row. Block-row G is computed by consumer warp G mod 8:
// lane l takes the tile columns j = l + 32 s (s < K) of all V rows, so a
// lane owns the same columns in every block-row, keeps their x values and
// their transposed partial sums in registers, and accumulates the V row
// sums, which the warp reduces once per block-row. Products are formed in
// pairs with the packed float32 FMA (fma.rn.f32x2). When the operator's
// last block-row is done the warps' transposed partials are summed in warp
// order in shared memory and added to the row sums: the result depends
// neither on the grid, nor on the stage size, nor on the block that ran the
// operator.
constexpr int kSymK = 4;   // at most 4 x 32 tile columns: n <= 128 V
constexpr int kSymSmemCap = 200 * 1024;
constexpr int kSymMinStages = 2;   // shared-memory ring of the symmetric GEMV: 2 to 8 stages
constexpr int kSymMaxStages = 8;
constexpr int kSymStages = 4;      // the deepest ring the tuning may choose (the support check assumes it)


// Packed pairs of float32 values (fma.rn.f32x2, sm_100 and later).
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ float f2_sum(uint64_t v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return lo + hi;
}
// One 16-byte operator vector as V / 2 pairs of float32 values.
template <typename T> struct SymVec;
template <> struct SymVec<float> {
  static constexpr int P = 2;
  __device__ static void load(const float* p, uint64_t (&o)[2]) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};
template <> struct SymVec<__nv_bfloat16> {
  static constexpr int P = 4;
  __device__ static void load(const __nv_bfloat16* p, uint64_t (&o)[4]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = f2_pack(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
  }
};

// Sums of V values over the 32 lanes: log2(V) halving exchanges (the lanes
// with the exchange bit set keep the upper half), then full ones. Afterwards
// lane l holds in v[0] the total of value sym_row(l).
template <int V>
__device__ __forceinline__ float warp_sum_rows(float (&v)[V], int lane) {
#pragma unroll
  for (int o = 16, n = V; n > 1; o >>= 1, n >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float send = upper ? v[i] : v[i + n / 2];
      const float keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 16 / V; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}
template <int V>
__device__ __forceinline__ int sym_row(int lane) {
  int q = 0;
#pragma unroll
  for (int o = 16, n = V; n > 1; o >>= 1, n >>= 1) q = 2 * q + ((lane & o) != 0);
  return q;
}

// One 16-byte vector from shared memory (32-bit shared-space address) as
// V / 2 pairs of float32 values.
template <typename T> struct SymLds;
template <> struct SymLds<float> {
  __device__ static void load(uint32_t addr, uint64_t (&o)[2]) {
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(o[0]), "=l"(o[1]) : "r"(addr));
  }
};
template <> struct SymLds<__nv_bfloat16> {
  __device__ static void load(uint32_t addr, uint64_t (&o)[4]) {
    uint32_t w[4];
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "r"(addr));
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = f2_pack(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
  }
};

// R rows of one block-row against the lane's NS active tile slots.
// ad[s] / st[s]: shared address of the lane's vector in the first row and
// the row pitch in bytes, or the address of a zero vector and 0 for a lane
// with no tile in slot s (its products are then 0). Rows from nr on are
// absent (the last block-row of an operator); PARTIAL selects the check.
template <typename T, int K, int NS, int R, bool PARTIAL>
__device__ __forceinline__ void sym_rows(uint32_t (&ad)[K], const uint32_t (&st)[K], const float* xrow, int nr,
                                         const uint64_t (&xj)[K][SymVec<T>::P],
                                         uint64_t (&accT)[K][SymVec<T>::P], float (&rs)[R]) {
  constexpr int P = SymVec<T>::P;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    rs[r] = 0.0f;
    if (!PARTIAL || r < nr) {
      const float xr = xrow[r];
      const uint64_t xrr = f2_pack(xr, xr);
      uint64_t racc = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        uint64_t a[P];
        SymLds<T>::load(ad[s], a);
        ad[s] += st[s];
#pragma unroll
        for (int i = 0; i < P; ++i) {
          racc = f2_fma(a[i], xj[s][i], racc);
          accT[s][i] = f2_fma(a[i], xrr, accT[s][i]);
        }
      }
      rs[r] = f2_sum(racc);
    }
  }
}
// Rows of one warp unit: a whole block-row (splitting BF16 block-rows over
// two warps was measured 9 % slower on GB300).
template <typename T> struct SymUnit { static constexpr int R = Op<T>::V; };

template <typename T, int K>
__global__ void __launch_bounds__(kTmaThreads) __maxnreg__(K <= 2 ? 72 : 96)
    k_sgemv_tma(const WorkItem* __restrict__ items, int n_items, const T* __restrict__ arena,
                const double* __restrict__ X, double* __restrict__ Y, const int32_t* __restrict__ yscatter,
                int stage_bytes, int nst, int max_n, int32_t* __restrict__ err) {
  constexpr int V = Op<T>::V;
  constexpr int P = SymVec<T>::P;   // float pairs per 16-byte vector
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int nx = 32 * K * V;                 // x as float, padded to whole lane slots
  const int npad = (max_n + V - 1) / V * V;      // x (float64), row sums, transposed partials
  unsigned char* stages = smem;
  float* xs = reinterpret_cast<float*>(smem + (size_t)nst * stage_bytes);
  double* xraw = reinterpret_cast<double*>(xs + nx);
  float* rowp = reinterpret_cast<float*>(xraw + npad);
  float* red = rowp + npad;
  uint64_t* full = reinterpret_cast<uint64_t*>(red + (size_t)kConsumerWarps * npad);
  uint64_t* empty = full + nst;
  __shared__ int abort_flag;
  __shared__ int stage_end[kSymMaxStages];   // last block-row + 1 of the stage in each slot (written by the producer)
  __shared__ __align__(16) uint4 zvec;  // the vector a lane without a tile reads
  const int stage_elems = stage_bytes / (int)sizeof(T);
  const uint32_t zero_addr = smem_addr(&zvec);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    abort_flag = 0;
    zvec = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    int slot = 0;
    uint32_t phase = 0;
    bool pending[kSymMaxStages];
    uint32_t pend_parity[kSymMaxStages];
    for (int s = 0; s < kSymMaxStages; ++s) pending[s] = false;
    bool ok = true;
    for (int u = blockIdx.x; u < n_items && ok; u += gridDim.x) {
      const WorkItem w = items[u];
      const int n = w.ncols, nblk = (n + V - 1) / V;
      for (int G0 = 0, G1; G0 < nblk; G0 = G1) {
        G1 = sym_stage_end<V>(G0, nblk, n, stage_elems);
        if (!mbar_wait(&empty[slot], phase ^ 1u) || *(volatile int*)&abort_flag) {
          atomicExch(err, BDDC_ERR_TIMEOUT);
          abort_flag = 1;
          ok = false;
          break;
        }
        const int32_t e0 = blk_off<V>(G0, n), e1 = blk_off<V>(G1, n);
        const uint32_t bytes = (uint32_t)(e1 - e0) * (uint32_t)sizeof(T);
        stage_end[slot] = G1;   // published by the arrive below (release), read after the wait (acquire)
        mbar_expect_tx(&full[slot], bytes);
        bulk_load(stages + (size_t)slot * stage_bytes, arena + w.moff + e0, bytes, &full[slot]);

        pending[slot] = true;
        pend_parity[slot] = phase;
        if (++slot == nst) { slot = 0; phase ^= 1u; }
      }
    }
    for (int s = 0; s < nst; ++s)
      if (pending[s] && !mbar_wait(&full[s], pend_parity[s])) atomicExch(err, BDDC_ERR_TIMEOUT);
    return;
  }

  // ---------------- consumers ----------------
  constexpr int kCT = kConsumerWarps * 32;
  const int tid = threadIdx.x;
  int slot = 0;
  uint32_t phase = 0;
  bool aborted = false;
  auto prefetch_operand = [&](int uu) {
    const WorkItem wn = items[uu];
    for (int i = tid; i < npad; i += kCT) {
      if (i < wn.ncols)
        cp_async8(xraw + i, X + wn.xoff + i);
      else
        xraw[i] = 0.0;
    }
    cp_async_commit();
  };
  // Two block barriers per operator: after the operand of the first
  // operator has landed, each operator is computed, then (barrier A: all
  // partials written, the next operand landed) the result is summed while
  // the next operand is converted to float32, then (barrier B: xs complete,
  // the partials and xraw free) the operand after it is prefetched.
  auto convert_operand = [&]() {
    for (int i = tid; i < nx; i += kCT) xs[i] = i < npad ? (float)xraw[i] : 0.0f;
  };
  if (blockIdx.x < n_items) {
    prefetch_operand(blockIdx.x);
    cp_async_wait_all();
    consumer_sync();                          // operand landed
    convert_operand();
    consumer_sync();                          // xs complete; xraw free
    if (blockIdx.x + (int)gridDim.x < n_items) prefetch_operand(blockIdx.x + gridDim.x);
  }
  for (int u = blockIdx.x; u < n_items; u += gridDim.x) {
    const WorkItem w = items[u];
    const int n = w.ncols, nblk = (n + V - 1) / V;
    const bool has_next = u + (int)gridDim.x < n_items;
    // this lane's columns: tile columns j = lane + 32 s, x in pairs
    uint64_t xj[K][P], accT[K][P];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
      for (int i = 0; i < P; i += 2) {   // 16-byte loads: two pairs each
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(xs + (s * 32 + lane) * V + 2 * i);
        xj[s][i] = v.x;
        xj[s][i + 1] = v.y;
        accT[s][i] = 0;
        accT[s][i + 1] = 0;
      }
    for (int G0 = 0, G1; G0 < nblk; G0 = G1) {
      // every warp visits every stage in order, so that no warp reaches a
      // slot whose barriers are a whole phase behind the stage it wants
      if (!aborted && (*(volatile int*)&abort_flag || !mbar_wait(&full[slot], phase))) {
        if (lane == 0) atomicExch(err, BDDC_ERR_TIMEOUT);
        abort_flag = 1;
        aborted = true;
      }
      G1 = aborted ? sym_stage_end<V>(G0, nblk, n, stage_elems) : stage_end[slot];
      if (!aborted) {
        const uint32_t tile_addr = smem_addr(stages + (size_t)slot * stage_bytes);
        const int32_t base = blk_off<V>(G0, n);
        // warp units: rows [h R, h R + R) of block-row G, unit index G H + h,
        // dealt round-robin over the warps by that index
        constexpr int R = SymUnit<T>::R, H = V / R;
        const int U0 = G0 * H, U1 = G1 * H;
        for (int U = U0 + ((warp - U0 % kConsumerWarps + kConsumerWarps) % kConsumerWarps); U < U1;
             U += kConsumerWarps) {
          const int G = U / H, r0 = (U - G * H) * R;
          const int nr = min(V, n - V * G) - r0;        // rows of this unit (R but in the last block-row)
          if (nr <= 0) continue;
          const uint32_t pitch = (uint32_t)(G + 1) * 16u;  // bytes per row: G + 1 vectors
          const uint32_t row0 =
              tile_addr + (uint32_t)(blk_off<V>(G, n) - base) * (uint32_t)sizeof(T) + (uint32_t)r0 * pitch;
          uint32_t ad[K], st[K];
#pragma unroll
          for (int s = 0; s < K; ++s) {
            const int j = 32 * s + lane;
            ad[s] = j <= G ? row0 + 16u * (uint32_t)j : zero_addr;
            st[s] = j <= G ? pitch : 0u;
          }
          const float* xrow = xs + V * G + r0;          // zero beyond n
          const int ns = min(K, G / 32 + 1);            // tile slots with a tile of this block-row
          float rs[R];
          if (nr >= R) {
            if (K == 1 || ns == 1) sym_rows<T, K, 1, R, false>(ad, st, xrow, nr, xj, accT, rs);
            else if (K == 2 || ns == 2) sym_rows<T, K, (K >= 2 ? 2 : 1), R, false>(ad, st, xrow, nr, xj, accT, rs);
            else if (ns == 3) sym_rows<T, K, (K >= 3 ? 3 : 1), R, false>(ad, st, xrow, nr, xj, accT, rs);
            else sym_rows<T, K, K, R, false>(ad, st, xrow, nr, xj, accT, rs);
          } else {
            sym_rows<T, K, K, R, true>(ad, st, xrow, nr, xj, accT, rs);   // last block-row: all slots (zero vectors beyond)
          }
          const float tot = warp_sum_rows<R>(rs, lane);
          const int row = V * G + r0 + sym_row<R>(lane);
          if ((lane & (32 / R - 1)) == 0 && row < n) rowp[row] = tot;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
      if (++slot == nst) { slot = 0; phase ^= 1u; }
    }
    // the warps' transposed partials, summed in warp order, plus the row sums
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
      for (int i = 0; i < P; i += 2) {   // 16-byte stores: two pairs each
        const int c = (s * 32 + lane) * V + 2 * i;
        if (c < npad) *reinterpret_cast<ulonglong2*>(red + (size_t)warp * npad + c) = make_ulonglong2(accT[s][i], accT[s][i + 1]);
      }
    cp_async_wait_all();                      // this thread's copies of the next operand landed
    consumer_sync();                          // A: partials and row sums written; xs no longer read
    if (!aborted)
      for (int c = tid; c < n; c += kCT) {
        float y = rowp[c];
#pragma unroll
        for (int ww = 0; ww < kConsumerWarps; ++ww) y += red[(size_t)ww * npad + c];
        const int64_t jy = (int64_t)w.yoff + c;
        Y[yscatter ? (int64_t)yscatter[jy] : jy] = (double)y;
      }
    if (has_next) convert_operand();
    consumer_sync();                          // B: xs complete; red, rowp and xraw free
    if (u + 2 * (int)gridDim.x < n_items) prefetch_operand(u + 2 * gridDim.x);
  }
  cp_async_wait_all();
}

template <typename T, int K>
size_t sym_smem(int stage_bytes, int nst, int max_n) {
  constexpr int V = Op<T>::V;
  const int npad = (max_n + V - 1) / V * V;
  return (size_t)nst * stage_bytes + (size_t)32 * K * V * 4 + (size_t)npad * (8 + 4 + 4 * kConsumerWarps) +
         2 * (size_t)nst * sizeof(uint64_t);
}

// Bytes of the widest block-row (V rows of the longest row), rounded up to
// 128: the smallest stage.
template <typename T>
int64_t sym_min_stage(int max_n) {
  constexpr int V = Op<T>::V;
  const int64_t q = (max_n + V - 1) / V;
  return (q * V * V * (int64_t)sizeof(T) + 127) / 128 * 128;
}

template <typename T, int K>
cudaError_t run_sym(const WorkItem* items, int n_items, int max_n, const T* arena, const double* X, double* Y,
                    const int32_t* yscatter, int32_t* err, cudaStream_t st, int stage_kb, int nst, int max_per_sm) {
  // a stage holds at least one whole block-row (the widest), and the
  // block's shared memory stays within kSymSmemCap
  const int64_t minst = sym_min_stage<T>(max_n);
  const int64_t room = ((int64_t)kSymSmemCap - (int64_t)sym_smem<T, K>(0, nst, max_n)) / nst / 128 * 128;
  const int64_t want = ((int64_t)stage_kb * 1024 + 127) / 128 * 128;
  const int stage_bytes = (int)std::max<int64_t>(minst, std::min<int64_t>(want, room));
  const size_t smem = sym_smem<T, K>(stage_bytes, nst, max_n);
  if (smem > (size_t)kSymSmemCap) return cudaErrorInvalidValue;
  auto kern = k_sgemv_tma<T, K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaThreads, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, per_sm);
  if (max_per_sm > 0) per_sm = std::min(per_sm, max_per_sm);
  const int grid = std::max(1, std::min(n_items, num_sms() * per_sm));
  kern<<<grid, kTmaThreads, smem, st>>>(items, n_items, arena, X, Y, yscatter, stage_bytes, nst, max_n, err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_sym(const WorkItem* items, int n_items, int max_n, const void* arena, const double* X,
                         double* Y, const int32_t* yscatter, int32_t* err, cudaStream_t st, int stage_kb,
                         int nst, int max_per_sm) {
  constexpr int V = Op<T>::V;
  const T* A = static_cast<const T*>(arena);
  if (max_n <= 32 * V)
    return run_sym<T, 1>(items, n_items, max_n, A, X, Y, yscatter, err, st, stage_kb, nst, max_per_sm);
  if (max_n <= 64 * V)
    return run_sym<T, 2>(items, n_items, max_n, A, X, Y, yscatter, err, st, stage_kb, nst, max_per_sm);
  if (max_n <= kSymK * 32 * V)
    return run_sym<T, kSymK>(items, n_items, max_n, A, X, Y, yscatter, err, st, stage_kb, nst, max_per_sm);
  return cudaErrorInvalidValue;
}

}  // namespace

bool bgemv_tma_supported(int precision, int max_lda) {
  const size_t eb = precision == BDDC_PREC_FP64 ? 8 : precision == BDDC_PREC_FP32 ? 4 : 2;
  const size_t xb = precision == BDDC_PREC_FP64   ? x_bytes<double, 1>(max_lda)
                    : precision == BDDC_PREC_FP32 ? x_bytes<float, 1>(max_lda)
                                                  : x_bytes<__nv_bfloat16, 1>(max_lda);
  const size_t row = ((size_t)max_lda * eb + 127) / 128 * 128;
  return kStages * row + xb + 64 <= 200 * 1024;
}

int64_t sym_packed_elems(int precision, int n) {
  return precision == BDDC_PREC_FP32 ? tri_off<4>(n) : tri_off<8>(n);
}

bool sgemv_tma_supported(int precision, int max_n) {
  if (precision != BDDC_PREC_FP32 && precision != BDDC_PREC_BF16) return false;
  const int V = precision == BDDC_PREC_FP32 ? 4 : 8;
  if (max_n > kSymK * 32 * V) return false;
  // the smallest stage: one whole block-row
  const size_t smem = precision == BDDC_PREC_FP32
                          ? sym_smem<float, kSymK>((int)sym_min_stage<float>(max_n), kSymStages, max_n)
                          : sym_smem<__nv_bfloat16, kSymK>((int)sym_min_stage<__nv_bfloat16>(max_n), kSymStages, max_n);
  return smem <= (size_t)kSymSmemCap;
}

cudaError_t launch_sgemv_tma(int precision, const WorkItem* items, int n_items, int max_n, const void* arena,
                             const double* X, double* Y, const int32_t* yscatter, int32_t* err, cudaStream_t st,
                             int stage_kb, int n_stages, int max_per_sm) {
  if (n_items == 0) return cudaSuccess;
  if (stage_kb < 1 || stage_kb > 48 || n_stages < kSymMinStages || n_stages > kSymMaxStages)
    return cudaErrorInvalidValue;
  if (precision == BDDC_PREC_FP32)
    return dispatch_sym<float>(items, n_items, max_n, arena, X, Y, yscatter, err, st, stage_kb, n_stages,
                               max_per_sm);
  if (precision == BDDC_PREC_BF16)
    return dispatch_sym<__nv_bfloat16>(items, n_items, max_n, arena, X, Y, yscatter, err, st, stage_kb, n_stages,
                                       max_per_sm);
  return cudaErrorInvalidValue;
}

cudaError_t launch_bgemv_tma(int precision, const WorkItem* items, int n_items, int max_lda, const void* arena,
                             const double* X, double* Y, const int32_t* yscatter, int nrhs, int32_t* err,
                             cudaStream_t st, int stage_kb, int max_per_sm) {
  if (n_items == 0) return cudaSuccess;
  if (stage_kb < 1 || stage_kb > 64) return cudaErrorInvalidValue;
  switch (precision) {
    case BDDC_PREC_FP64:
      return dispatch<double>(items, n_items, max_lda, arena, X, Y, yscatter, nrhs, err, st, stage_kb, max_per_sm);
    case BDDC_PREC_FP32:
      return dispatch<float>(items, n_items, max_lda, arena, X, Y, yscatter, nrhs, err, st, stage_kb, max_per_sm);
    default:
      return dispatch<__nv_bfloat16>(items, n_items, max_lda, arena, X, Y, yscatter, nrhs, err, st, stage_kb, max_per_sm);
  }
}

}  // namespace bddc
