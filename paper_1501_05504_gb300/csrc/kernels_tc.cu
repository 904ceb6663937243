// Tensor-core grouped GEMM for sm_103a (tcgen05, TMEM accumulators).
//
// Same task tables as the FP64 kernel (one output block per task, K-segments
// summed), computed on the 5th-generation tensor cores in TF32 with FP32
// accumulation per 32-wide K chunk and double-float accumulation across
// chunks.  Operands are FP64 tensors pre-split into x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi) (Ootomo and Yokota's split, 2022) by
// split_kernel or by the MPO combination, so the GEMM itself does no FP64
// arithmetic (GB300's FP64 rate is ~1/1000 of its TF32 rate):
//   kPasses = 1: C = A_hi B_hi                                  (TF32)
//   kPasses = 3: C = A_hi B_hi + A_hi B_lo + A_lo B_hi          (3xTF32)
//
// CTA tile 128 x 64 (M x N), K chunks of 32, two shared-memory stages and two
// TMEM accumulator buffers.  All 128 threads load the operand tiles; one
// thread issues tcgen05.mma and commits each stage to an mbarrier; while the
// tensor core works on chunk k the four warps drain chunk k-1's FP32
// accumulator (tcgen05.ld) into double-float registers.  Each output element
// is stored as its (hi, lo) FP32 pair, for the double-float combinations that
// consume it.  Every wait on an mbarrier is bounded: on time-out the CTA
// records an error code, frees its tensor memory and returns.
#include <atomic>
#include <cstdint>

#include "kernels.hpp"

namespace dmrg3s {

namespace {

constexpr int TBM = 128, TBN = 64, TBK = 32, TNT = 128;
constexpr int kStageA = TBM * TBK * 4;            // bytes of one A tile (hi or lo)
constexpr int kStageB = TBN * TBK * 4;            // bytes of one B tile
constexpr uint32_t kTmemCols = 2 * TBN;          // two FP32 accumulator buffers
constexpr long long kSpinLimit = 1ll << 28;       // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Operand tiles use the K-major, non-swizzled canonical layout: core matrices
// of 8 rows x 16 bytes; element (row, k) at byte (row / 8) * 1024 +
// (k / 4) * 128 + (row % 8) * 16 + (k % 4) * 4, i.e. K-adjacent core matrices
// 128 B apart (leading byte offset) and 8-row groups 1024 B apart (stride
// byte offset).

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 1024;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split(double x, float& hi, float& lo) {
  hi = to_tf32((float)x);
  lo = to_tf32((float)(x - (double)hi));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Load one operand tile (ROWS x 32, K-major canonical layout) from the
// pre-split FP32 arrays.  kContig: the source is contiguous along K (element
// (row, k) at src[row * ld + k]); otherwise along the row index
// (src[k * ld + row]).  Lanes cover one 8 x 4 core matrix per step (a
// 128-byte contiguous shared store), with the fast lane index along the
// source's contiguous direction.  No FP64 arithmetic: GB300's FP64 rate would
// otherwise bound the kernel.
template <int ROWS, bool kContig, bool kLo>
__device__ __forceinline__ void load_tile(const float* __restrict__ shi, const float* __restrict__ slo,
                                          int ld, int row0, int nrow, int k0, int nk,
                                          unsigned char* hi, unsigned char* lo, int warp,
                                          int lane) {
  const int r8 = kContig ? (lane >> 2) : (lane & 7);
  const int k4 = kContig ? (lane & 3) : (lane >> 3);
#pragma unroll
  for (int g = warp; g < ROWS / 8; g += 4) {
    const int row = g * 8 + r8;
    const bool rok = row0 + row < nrow;
    float vh[8], vl[8];
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      const int k = k0 + kc * 4 + k4;
      const int64_t o = kContig ? (int64_t)(row0 + row) * ld + k : (int64_t)k * ld + row0 + row;
      const bool ok = rok && k < nk;
      vh[kc] = ok ? shi[o] : 0.f;
      if (kLo) vl[kc] = ok ? slo[o] : 0.f;
    }
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      const uint32_t o = (uint32_t)(g * 1024 + kc * 128 + r8 * 16 + k4 * 4);
      *reinterpret_cast<float*>(hi + o) = vh[kc];
      if (kLo) *reinterpret_cast<float*>(lo + o) = vl[kc];
    }
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Add the FP32 accumulator of one K chunk (TMEM columns col0 .. col0 + 63 of
// this warp's lanes) into the thread's double-float accumulators (hi, lo),
// with Knuth's two-sum so that no rounding error is lost between chunks.
__device__ __forceinline__ void drain(uint32_t dtmem, int warp, uint32_t col0, float (&ah)[TBN],
                                      float (&al)[TBN]) {
#pragma unroll
  for (int c0 = 0; c0 < TBN; c0 += 16) {
    uint32_t v[16];
    tmem_ld16(dtmem + ((uint32_t)(warp * 32) << 16) + col0 + (uint32_t)c0, v);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float x = __uint_as_float(v[j]), a = ah[c0 + j];
      const float s = __fadd_rn(a, x);
      const float bb = __fsub_rn(s, a);
      const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(x, bb));
      ah[c0 + j] = s;
      al[c0 + j] = __fadd_rn(al[c0 + j], e);
    }
  }
}

// Every 32-wide K chunk is accumulated by the tensor core into its own FP32
// TMEM buffer (two buffers, alternating) and then added into double-float
// registers, so FP32 rounding only ever sees 32-term sums.
template <Trans TA, Trans TB, int kPasses>
__global__ void __launch_bounds__(TNT, 2)
    gemm_tc_kernel(const GemmTile* __restrict__ tiles, const GemmTask* __restrict__ tasks,
                   const GemmSeg* __restrict__ segs, const float* __restrict__ Ahi,
                   const float* __restrict__ Alo, const float* __restrict__ Bhi,
                   const float* __restrict__ Blo, float2* __restrict__ C, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr bool kLo = kPasses == 3;
  constexpr int kStage = (kStageA + kStageB) * (kLo ? 2 : 1);
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const GemmTile tile = tiles[blockIdx.x];
  const GemmTask task = tasks[tile.task];
  const int m0 = tile.tm * TBM, n0 = tile.tn * TBN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t dtmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(TBM, TBN);
  float ah[TBN], al[TBN];
#pragma unroll
  for (int j = 0; j < TBN; ++j) {
    ah[j] = 0.f;
    al[j] = 0.f;
  }
  bool ok = true;
  int it = 0;

  for (int sgi = 0; sgi < task.nseg && ok; ++sgi) {
    const GemmSeg sg = segs[task.seg0 + sgi];
    for (int k0 = 0; k0 < sg.K; k0 += TBK, ++it) {
      const int st = it & 1;
      // stage st and TMEM buffer st were last used by chunk it - 2
      if (it >= 2 && ok) ok = mbar_wait(&bars[st], (uint32_t)(((it - 2) >> 1) & 1));
      unsigned char* base = smem + st * kStage;
      unsigned char* a_hi = base;
      unsigned char* a_lo = base + kStageA;
      unsigned char* b_hi = base + kStageA * (kLo ? 2 : 1);
      unsigned char* b_lo = b_hi + kStageB;
      load_tile<TBM, TA == Trans::N, kLo>(Ahi + sg.offA, kLo ? Alo + sg.offA : nullptr, sg.lda, m0,
                                          task.M, k0, sg.K, a_hi, a_lo, warp, lane);
      load_tile<TBN, TB == Trans::T, kLo>(Bhi + sg.offB, kLo ? Blo + sg.offB : nullptr, sg.ldb, n0,
                                          task.N, k0, sg.K, b_hi, b_lo, warp, lane);
      // make the generic-proxy stores visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      // one decision for the whole CTA (a wait that timed out in any thread
      // stops every thread), so that all threads meet the same barriers; a
      // stage written after a failed wait is never handed to the tensor core
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sah = smem_u32(a_hi), sal = smem_u32(a_lo);
        const uint32_t sbh = smem_u32(b_hi), sbl = smem_u32(b_lo);
        const uint32_t d = dtmem + (uint32_t)(st * TBN);
#pragma unroll
        for (int kk = 0; kk < TBK / 8; ++kk) {       // K = 8 per instruction (32 bytes)
          const uint32_t off = kk * 256;             // two core matrices along K
          if (kLo) {
            mma_tf32(d, smem_desc(sal + off), smem_desc(sbh + off), idesc, kk == 0 ? 0u : 1u);
            mma_tf32(d, smem_desc(sah + off), smem_desc(sbl + off), idesc, 1u);
            mma_tf32(d, smem_desc(sah + off), smem_desc(sbh + off), idesc, 1u);
          } else {
            mma_tf32(d, smem_desc(sah + off), smem_desc(sbh + off), idesc, kk == 0 ? 0u : 1u);
          }
        }
        mma_commit(&bars[st]);
      }
      // meanwhile drain the previous chunk's accumulator
      if (it >= 1) {
        ok = mbar_wait(&bars[(it - 1) & 1], (uint32_t)(((it - 1) >> 1) & 1));
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          drain(dtmem, warp, (uint32_t)(((it - 1) & 1) * TBN), ah, al);
        }
      }
    }
    ok = __syncthreads_and(ok);
  }
  // the last chunk
  if (ok && it > 0) {
    ok = mbar_wait(&bars[(it - 1) & 1], (uint32_t)(((it - 1) >> 1) & 1));
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      drain(dtmem, warp, (uint32_t)(((it - 1) & 1) * TBN), ah, al);
    }
  }
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    // ---- epilogue: thread (warp, lane) owns accumulator row 32 warp + lane
    const int gm = m0 + warp * 32 + lane;
    if (gm < task.M) {
      float2* crow = C + task.offC + (int64_t)gm * task.ldc + n0;
      const int nv = task.N - n0 < TBN ? task.N - n0 : TBN;
#pragma unroll
      for (int j = 0; j < TBN; ++j)
        if (j < nv) crow[j] = make_float2(ah[j], al[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtmem),
                 "r"(kTmemCols)
                 : "memory");
}

__global__ void split_kernel(const double* __restrict__ x, float* __restrict__ hi,
                             float* __restrict__ lo, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float h, l;
    split(x[i], h, l);
    hi[i] = h;
    if (lo) lo[i] = l;
  }
}

template <Trans TA, Trans TB, int P>
void launch_one(const GemmTile* tiles, int ntiles, const GemmTask* tasks, const GemmSeg* segs,
                const float* Ah, const float* Al, const float* Bh, const float* Bl, float2* C,
                int* err, cudaStream_t st) {
  constexpr int kLo = P == 3 ? 1 : 0;
  constexpr int smem = 2 * (kStageA + kStageB) * (1 + kLo);
  // the shared-memory limit is a per-device attribute of the kernel
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(done.load() & bit)) {
    cudaFuncSetAttribute(gemm_tc_kernel<TA, TB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    if (bit) done.fetch_or(bit);
  }
  gemm_tc_kernel<TA, TB, P><<<ntiles, TNT, smem, st>>>(tiles, tasks, segs, Ah, Al, Bh, Bl, C, err);
}

}  // namespace

void launch_split(const double* x, float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  int64_t g = (n + 255) / 256;
  if (g > 4 * 152) g = 4 * 152;
  split_kernel<<<(int)g, 256, 0, st>>>(x, hi, lo, n);
}

void launch_gemm_tc(int passes, Trans ta, Trans tb, const GemmTile* tiles, int ntiles,
                    const GemmTask* tasks, const GemmSeg* segs, const float* Ahi,
                    const float* Alo, const float* Bhi, const float* Blo, float2* C, int* err,
                    cudaStream_t st) {
  if (ntiles <= 0) return;
  count_launch();
#define DMRG3S_TC(TA_, TB_)                                                           \
  if (ta == Trans::TA_ && tb == Trans::TB_) {                                         \
    if (passes == 3)                                                                  \
      launch_one<Trans::TA_, Trans::TB_, 3>(tiles, ntiles, tasks, segs, Ahi, Alo, Bhi, Blo, C, \
                                            err, st);                                   \
    else                                                                              \
      launch_one<Trans::TA_, Trans::TB_, 1>(tiles, ntiles, tasks, segs, Ahi, Alo, Bhi, Blo, C, \
                                            err, st);                                   \
    return;                                                                           \
  }
  DMRG3S_TC(N, N)
  DMRG3S_TC(N, T)
  DMRG3S_TC(T, N)
  DMRG3S_TC(T, T)
#undef DMRG3S_TC
}

}  // namespace dmrg3s
