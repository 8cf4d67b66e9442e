// Tensor-core batched GEMM for blocks of right-hand sides (sm_103a): the
// local operators of the apply (A_II^-1 and K_GG of every subdomain, Sec. 2)
// times an nrhs-column operand, Y = Op X, with tcgen05.mma accumulating in
// tensor memory and the operator streamed from HBM once per launch.
//
// Operands. BF16 operators use kind::f16; FP32 operators use kind::tf32
// (the tensor core reads them as TF32). The float64 operand x is split into
// a high and a low part in the operator's format, x ~ hi + lo (about 16
// significant bits for BF16, 21 for TF32), and every K step issues two MMAs
// into the same float32 accumulator, so the operand is not rounded to the
// operator's precision.
//
// Layout. Operators are stored by tc_pack_host (setup) as chunks of up to
// 128 rows x 128 bytes of columns in the canonical no-swizzle K-major layout:
// core matrices of 8 rows x 16 bytes ordered [8-row group][16-byte column
// slice][8 rows][16 bytes]. The valid rows of a chunk are a contiguous prefix,
// so a partial row tile costs no padding in HBM (the rows beyond it produce
// accumulator lanes that are never read). The packed operand uses the same
// layout with the right-hand sides as rows.
//
// Per launch:
//   k_tc_pack  X (float64, compact, nrhs per row) -> hi/lo operand chunks.
//   k_tc_gemm  persistent, one CTA per SM, 6 warps. Warp 0 lane 0 issues the
//              bulk copies (per column chunk: the operand chunk, then the
//              unit's operator chunks), warp 1 owns tensor memory and its lane
//              0 issues the MMAs, warps 2-5 read the accumulators with
//              tcgen05.ld and write Y in float64. A unit is up to 8 row tiles
//              of one operator, so an operand chunk is loaded once per 8 tiles.
// Every mbarrier wait is bounded. On timeout the kernel records
// BDDC_ERR_TIMEOUT, stops issuing work, waits (bounded) for its copies and
// MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace bddc {

namespace {

constexpr int kThreadsTc = 192;                 // 6 warps
constexpr int kAStages = 6;
constexpr int kBStages = 2;
constexpr int kChunkBytes = kTcRows * 128;      // 16 KB operator chunk
constexpr int kBStageBytes = 2 * 64 * 128;      // hi + lo, up to 64 right-hand sides
constexpr int kSmemA = kAStages * kChunkBytes;
constexpr int kSmemB = kBStages * kBStageBytes;
constexpr int kNumBars = 2 * kAStages + 2 * kBStages + 5;
constexpr int kSmemTc = kSmemA + kSmemB + kNumBars * 8 + 16;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

template <typename T> struct TcFmt;
template <> struct TcFmt<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;   // instruction descriptor A/B format: BF16 (kind::f16)
};
template <> struct TcFmt<float> {
  static constexpr uint32_t fmt = 2;   // TF32 (kind::tf32)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
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
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, the
// byte distance between core matrices adjacent in K (leading) and in M/N
// (stride), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor: float32 accumulator, A and B of the given format,
// both K-major, N columns, M = 128 rows.
__host__ __device__ __forceinline__ uint32_t idesc(uint32_t fmt, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

template <typename T>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
  if constexpr (sizeof(T) == 2)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
// Arrive (once) on bar when every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x ~ hi + lo in the operator's format.
__device__ __forceinline__ void split(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  const float f = (float)x;
  hi = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}
__device__ __forceinline__ void split(double x, float& hi, float& lo) {
  const float f = (float)x;
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
  hi = __uint_as_float(h);
  lo = f - hi;
}
__device__ __forceinline__ uint32_t bits(__nv_bfloat16 v) { return (uint32_t)__bfloat16_as_ushort(v); }
__device__ __forceinline__ uint32_t bits(float v) { return __float_as_uint(v); }

}  // namespace

// Operator columns padded to the MMA K step (32 bytes).
__host__ __device__ inline int tc_kpad(int n, int esz) {
  const int ks = 32 / esz;
  return (n + ks - 1) / ks * ks;
}

namespace {

// Packed operand: per operator, per column chunk kc (128 bytes of columns,
// the last one narrower), a hi block then a lo block, each
// [N/8 row groups][kw/EPS slices][8 right-hand sides][16 bytes]. One thread
// writes one 16-byte vector of hi and of lo (EPS consecutive columns of one
// right-hand side).
template <typename T>
__global__ void __launch_bounds__(256) k_tc_pack(const int32_t* __restrict__ slice_op, int64_t n_slices,
                                                 const int32_t* __restrict__ opinfo, const double* __restrict__ X,
                                                 int nrhs, int N, unsigned char* __restrict__ Bp) {
  constexpr int esz = (int)sizeof(T), EPS = 16 / esz, KCH = 128 / esz;
  const int64_t total = n_slices * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / N;
    const int nn = (int)(t - q * N);
    const int op = slice_op[q];
    const int xoff = opinfo[4 * op], n = opinfo[4 * op + 1], kbase = opinfo[4 * op + 2], slice0 = opinfo[4 * op + 3];
    const int c0 = (int)(q - slice0) * EPS;
    const int kc = c0 / KCH, j = (c0 - kc * KCH) / EPS;
    const int kw = min(KCH, tc_kpad(n, esz) - kc * KCH), nsl = kw / EPS;
    unsigned char* chunk = Bp + ((int64_t)kbase * 2 * N + (int64_t)kc * 2 * N * KCH) * esz;
    const int64_t off = ((int64_t)(nn >> 3) * nsl + j) * 128 + (nn & 7) * 16;
    uint32_t hw[4] = {0, 0, 0, 0}, lw[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < EPS; ++e) {
      const int c = c0 + e;
      const double x = (c < n && nn < nrhs) ? X[(int64_t)(xoff + c) * nrhs + nn] : 0.0;
      T h, l;
      split(x, h, l);
      const int word = e * esz / 4, shift = (e * esz % 4) * 8;
      hw[word] |= bits(h) << shift;
      lw[word] |= bits(l) << shift;
    }
    *reinterpret_cast<uint4*>(chunk + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(chunk + (int64_t)N * kw * esz + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsTc, 1)
    k_tc_gemm(const TcUnit* __restrict__ units, int n_units, const T* __restrict__ arena,
              const unsigned char* __restrict__ Bp, double* __restrict__ Y, const int32_t* __restrict__ yscatter,
              int nrhs, int N, int nbuf, int32_t* __restrict__ err) {
  constexpr int esz = (int)sizeof(T), EPS = 16 / esz, KCH = 128 / esz, KSTEP = 2 * EPS;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + kSmemA;
  uint64_t* a_full = reinterpret_cast<uint64_t*>(smem + kSmemA + kSmemB);
  uint64_t* a_empty = a_full + kAStages;
  uint64_t* b_full = a_empty + kAStages;
  uint64_t* b_empty = b_full + kBStages;
  uint64_t* acc_full = b_empty + kBStages;   // [2]: accumulator buffer b complete
  uint64_t* acc_empty = acc_full + 2;        // [2]: accumulator buffer b read out
  uint64_t* fin = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kAStages; ++s) { mbar_init(&a_full[s], 1); mbar_init(&a_empty[s], 1); }
    for (int s = 0; s < kBStages; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 4); }
    mbar_init(fin, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    atomicExch(err, BDDC_ERR_TIMEOUT);
    *(volatile int*)&abort_flag = 1;
  };
  auto aborted = [&]() { return *(volatile int*)&abort_flag != 0; };

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const TcUnit w = units[u];
        const int kpad = tc_kpad(w.n, esz);
        const int nkc = (kpad + KCH - 1) / KCH;
        const unsigned char* asrc = reinterpret_cast<const unsigned char*>(arena) + w.aoff * esz;
        const unsigned char* bsrc = Bp + (int64_t)w.kbase * 2 * N * esz;
        for (int kc = 0; kc < nkc && ok; ++kc) {
          const int kw = min(KCH, kpad - kc * KCH);
          if (!mbar_wait(&b_empty[bs], bph ^ 1u) || aborted()) { fail(); ok = false; break; }
          const uint32_t bbytes = (uint32_t)(2 * N * kw * esz);
          mbar_expect_tx(&b_full[bs], bbytes);
          bulk_load(sB + bs * kBStageBytes, bsrc + (int64_t)kc * 2 * N * KCH * esz, bbytes, &b_full[bs]);
          if (++bs == kBStages) { bs = 0; bph ^= 1u; }
          for (int mt = 0; mt < w.g; ++mt) {
            const int nr = min(kTcRows, w.n - (w.row0 + mt * kTcRows));
            const uint32_t abytes = (uint32_t)(((nr + 7) & ~7) * kw * esz);
            if (!mbar_wait(&a_empty[as], aph ^ 1u) || aborted()) { fail(); ok = false; break; }
            mbar_expect_tx(&a_full[as], abytes);
            bulk_load(sA + as * kChunkBytes, asrc, abytes, &a_full[as]);
            asrc += abytes;
            if (++as == kAStages) { as = 0; aph ^= 1u; }
          }
        }
      }
      // the copies in flight land before the block exits: after the last
      // use of every stage its consumer releases it (or a wait runs out)
      for (int s = 0; s < kAStages; ++s) {
        if (!mbar_wait(&a_empty[as], aph ^ 1u)) { fail(); break; }
        if (++as == kAStages) { as = 0; aph ^= 1u; }
      }
      for (int s = 0; s < kBStages; ++s) {
        if (!mbar_wait(&b_empty[bs], bph ^ 1u)) { fail(); break; }
        if (++bs == kBStages) { bs = 0; bph ^= 1u; }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id = idesc(TcFmt<T>::fmt, N);
      int as = 0, bs = 0, nunit = 0;
      uint32_t aph = 0, bph = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++nunit) {
        const TcUnit w = units[u];
        const int kpad = tc_kpad(w.n, esz);
        const int nkc = (kpad + KCH - 1) / KCH;
        // accumulators: nbuf buffers of 256 columns (or one of 512), used in turn
        const int ab = nunit % nbuf, use = nunit / nbuf;
        if (use > 0 && (!mbar_wait(&acc_empty[ab], (uint32_t)(use - 1) & 1u) || aborted())) { fail(); break; }
        tc_fence_after();
        for (int kc = 0; kc < nkc && ok; ++kc) {
          const int kw = min(KCH, kpad - kc * KCH), nsl = kw / EPS;
          const uint32_t sbo = (uint32_t)nsl * 128u;
          if (!mbar_wait(&b_full[bs], bph) || aborted()) { fail(); ok = false; break; }
          tc_fence_after();
          const uint32_t bst = smem_u32(sB + bs * kBStageBytes);
          const uint32_t blo = (uint32_t)(N * kw * esz);
          for (int mt = 0; mt < w.g; ++mt) {
            if (!mbar_wait(&a_full[as], aph) || aborted()) { fail(); ok = false; break; }
            tc_fence_after();
            const uint32_t ast = smem_u32(sA + as * kChunkBytes);
            const uint32_t d = tmem + (uint32_t)(ab * 256 + mt * N);
            for (int ks = 0; ks < kw / KSTEP; ++ks) {
              const uint64_t ad = sdesc(ast + ks * 256u, 128u, sbo);
              mma<T>(d, ad, sdesc(bst + ks * 256u, 128u, sbo), id, (kc | ks) != 0);
              mma<T>(d, ad, sdesc(bst + blo + ks * 256u, 128u, sbo), id, 1u);
            }
            mma_commit(&a_empty[as]);
            if (++as == kAStages) { as = 0; aph ^= 1u; }
          }
          mma_commit(&b_empty[bs]);
          if (++bs == kBStages) { bs = 0; bph ^= 1u; }
        }
        if (ok) mma_commit(&acc_full[ab]);
      }
      // every MMA issued has completed before tensor memory is freed
      mma_commit(fin);
      if (!mbar_wait(fin, 0u)) fail();
    }
  } else {
    // ---------------- epilogue: tensor memory -> Y ----------------
    const int quarter = warp & 3;   // this warp may read lanes [32 quarter, 32 quarter + 32)
    int nunit = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++nunit) {
      const TcUnit w = units[u];
      const int ab = nunit % nbuf, use = nunit / nbuf;
      bool ok = mbar_wait(&acc_full[ab], (uint32_t)use & 1u) && !aborted();
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      tc_fence_after();
      for (int mt = 0; mt < w.g; ++mt) {
        const int r = w.row0 + mt * kTcRows + quarter * 32 + lane;
        int64_t dst = -1;
        if (r < w.n) {
          const int64_t j = (int64_t)w.yoff + r;
          dst = yscatter ? (int64_t)yscatter[j] : j;
        }
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * 256 + mt * N + c0), v);
          if (dst >= 0) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (c0 + k < nrhs) Y[dst * nrhs + c0 + k] = (double)v[k];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

int g_sms_tc = 0;

}  // namespace

template <typename T>
void tc_pack_host(const std::vector<std::vector<double>>& ops, const std::vector<int>& dims,
                  const std::vector<int32_t>& xoff, TcPacked<T>& out) {
  constexpr int esz = (int)sizeof(T), EPS = 16 / esz, KCH = 128 / esz;
  out.arena.clear();
  out.units.clear();
  out.slice_op.clear();
  out.opinfo.clear();
  int64_t cur = 0, kbase = 0, slice0 = 0;
  for (size_t s = 0; s < ops.size(); ++s) {
    const int n = dims[s];
    const int kpad = n > 0 ? tc_kpad(n, esz) : 0;
    out.opinfo.insert(out.opinfo.end(), {xoff[s], n, (int32_t)kbase, (int32_t)slice0});
    if (n == 0) continue;
    const int nkc = (kpad + KCH - 1) / KCH, MT = (n + kTcRows - 1) / kTcRows;
    const double* M = ops[s].data();
    for (int gi = 0; gi < MT; gi += kTcGroup) {
      const int g = std::min(kTcGroup, MT - gi);
      out.units.push_back(TcUnit{cur, n, g, gi * kTcRows, xoff[s], xoff[s], (int32_t)kbase});
      for (int kc = 0; kc < nkc; ++kc) {
        const int kw = std::min(KCH, kpad - kc * KCH), nsl = kw / EPS;
        for (int mt = 0; mt < g; ++mt) {
          const int rt = (gi + mt) * kTcRows;
          const int rows8 = (std::min(kTcRows, n - rt) + 7) & ~7;
          out.arena.resize((size_t)(cur + (int64_t)rows8 * kw), TcCvt<T>::from(0.0));
          T* chunk = out.arena.data() + cur;
          for (int rg = 0; rg < rows8 / 8; ++rg)
            for (int j = 0; j < nsl; ++j)
              for (int r8 = 0; r8 < 8; ++r8) {
                const int row = rt + rg * 8 + r8;
                for (int e = 0; e < EPS; ++e) {
                  const int col = kc * KCH + j * EPS + e;
                  const double v = (row < n && col < n) ? M[(size_t)row * n + col] : 0.0;
                  chunk[((rg * nsl + j) * 8 + r8) * EPS + e] = TcCvt<T>::from(v);
                }
              }
          cur += (int64_t)rows8 * kw;
        }
      }
    }
    for (int q = 0; q < kpad / EPS; ++q) out.slice_op.push_back((int32_t)s);
    kbase += kpad;
    slice0 += kpad / EPS;
  }
  out.cols_total = kbase;
  out.max_g = 0;
  for (const TcUnit& u : out.units) out.max_g = std::max(out.max_g, u.g);
  if (out.arena.empty()) out.arena.push_back(TcCvt<T>::from(0.0));
  // largest units first: the persistent grid takes them round-robin
  std::stable_sort(out.units.begin(), out.units.end(), [&](const TcUnit& a, const TcUnit& b) {
    return (int64_t)a.g * tc_kpad(a.n, esz) > (int64_t)b.g * tc_kpad(b.n, esz);
  });
}

template void tc_pack_host<__nv_bfloat16>(const std::vector<std::vector<double>>&, const std::vector<int>&,
                                          const std::vector<int32_t>&, TcPacked<__nv_bfloat16>&);
template void tc_pack_host<float>(const std::vector<std::vector<double>>&, const std::vector<int>&,
                                  const std::vector<int32_t>&, TcPacked<float>&);

size_t tc_operand_bytes(int precision, int64_t cols_total, int nrhs_max) {
  const int esz = precision == BDDC_PREC_BF16 ? 2 : 4;
  const int64_t N = (nrhs_max + 15) / 16 * 16;
  return (size_t)std::max<int64_t>(cols_total, 1) * 2 * N * esz;
}

namespace {
template <typename T>
cudaError_t run_tc(bddc_handle_s* h, bool interior, const double* X, double* Y, const int32_t* yscatter, int nrhs,
                   cudaStream_t st) {
  const TcUnit* units = interior ? h->d_tcu_I : h->d_tcu_G;
  const int n_units = interior ? h->n_tcu_I : h->n_tcu_G;
  if (n_units == 0) return cudaSuccess;
  const int N = (nrhs + 15) / 16 * 16;
  const int64_t n_slices = interior ? h->n_tcs_I : h->n_tcs_G;
  const int64_t total = n_slices * N;
  const int pack_blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  k_tc_pack<T><<<pack_blocks, 256, 0, st>>>(interior ? h->d_tcs_I : h->d_tcs_G, n_slices,
                                           interior ? h->d_tcop_I : h->d_tcop_G, X, nrhs, N,
                                           static_cast<unsigned char*>(h->d_tcB));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto kern = k_tc_gemm<T>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc)) != cudaSuccess)
    return e;
  if (!g_sms_tc) {
    int dev;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms_tc, cudaDevAttrMultiProcessorCount, dev);
  }
  const int grid = std::max(1, std::min(n_units, g_sms_tc));
  // two accumulator buffers (the epilogue of one unit overlaps the MMAs of
  // the next) when every unit's tiles fit in half of tensor memory
  const int maxg = interior ? h->tc_maxg_I : h->tc_maxg_G;
  const int nbuf = maxg * N <= 256 ? 2 : 1;
  kern<<<grid, kThreadsTc, kSmemTc, st>>>(units, n_units, static_cast<const T*>(interior ? h->d_aii : h->d_kgg),
                                          static_cast<const unsigned char*>(h->d_tcB), Y, yscatter, nrhs, N, nbuf,
                                          h->d_err);
  h->launches += 2;
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tc_gemm(bddc_handle_s* h, bool interior, const double* X, double* Y, const int32_t* yscatter,
                           int nrhs, cudaStream_t st) {
  if (nrhs < 1 || nrhs > 64) return cudaErrorInvalidValue;
  return h->precision == BDDC_PREC_BF16 ? run_tc<__nv_bfloat16>(h, interior, X, Y, yscatter, nrhs, st)
                                        : run_tc<float>(h, interior, X, Y, yscatter, nrhs, st);
}

}  // namespace bddc
