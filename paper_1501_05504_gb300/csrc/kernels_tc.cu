// Tensor-core grouped GEMM for sm_103a (tcgen05, TMEM accumulators, bulk
// asynchronous copies), and the kernels that pack its operands.
//
// Operands are FP64 tensors split into x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi) (Ootomo and Yokota's split, 2022) and packed in tiles of
// 8 rows x 32 k in the K-major core-matrix order of the shared-memory matrix
// descriptors (kernels.hpp).  A 128-row slab of one 32-wide k-chunk is then a
// contiguous 16 KB run, so each operand slab reaches shared memory with one
// bulk copy (cp.async.bulk, completion counted in bytes on an mbarrier); no
// thread touches operand data on its way to the tensor core.
//
// Products per k-chunk of one 128 x 128 output tile:
//   kPasses = 1: D_main += A_hi B_hi                                (TF32)
//   kPasses = 3: D_main += A_hi B_hi,  D_corr += A_hi B_lo + A_lo B_hi  (3xTF32)
// The small correction terms keep their own TMEM accumulator over the whole
// K range (their FP32 rounding is ~2^-11 below the result).  The main
// accumulator is drained every kSpan k-chunks (128 k for kSpan = 4: 16
// accumulations of hi * hi products) into double-float registers with
// Knuth's two-sum, so FP32 rounding only ever sees a short span of main
// products.  The 512 TMEM columns hold two main and two correction buffers
// (four main buffers for TF32), so the tensor core can start the next tile
// while the drain warps still finish and store the previous one.  The last N
// tile of a block issues the narrowest MMA width (a multiple of 16) that
// covers it.  No FP64 instruction runs in the kernel (GB300's FP64 rate is
// ~1/1000 of its TF32 rate).
//
// Warp roles of the persistent CTA (one per SM, 384 threads = 3 warpgroups):
//   warp 0     one lane issues the bulk copies into a 3-stage shared-memory ring
//   warp 1     owns the tensor memory; one lane issues tcgen05.mma and commits
//              each stage and each accumulator to mbarriers
//   warps 2-3  idle (their warpgroup hands its registers to the drain warps)
//   warps 4-11 drain: warp w reads TMEM lanes 32 (w % 4) .. +31 (its row
//              quarter) and columns 64 ((w - 4) / 4) .. +63 of every tile, keeps
//              their double-float sums (128 registers) and stores the tile
//              through a small shared-memory transpose (coalesced rows of
//              (hi, lo) pairs).
// The CTA starts with 168 registers per thread (384 x 168 = 64,512 of the
// SM's 65,536); warpgroup 0 gives up to 56 (setmaxnreg.dec) and the two drain
// warpgroups take 224 (setmaxnreg.inc): 128 x 56 + 256 x 224 = 64,512.
// Units (output tiles) come in one list per CTA, balanced by the planner.
//
// Every wait on an mbarrier is bounded by the elapsed %globaltimer time given
// by the host.  A wait that runs out sets the device error word and a shared
// abort flag that every other wait also watches; all roles then leave their
// loops, the copy lane waits for its copies still in flight, the MMA lane for
// its products (a fixed one-second limit for these drains), and the CTA frees
// its tensor memory and returns.  Nothing traps.
#include <atomic>
#include <cstdint>

#include "kernels.hpp"

namespace dmrg3s {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 32;
constexpr int kStages = 3;
constexpr int kThreads = 384;                       // 12 warps
constexpr int kFirstDrainWarp = 4;
constexpr int kDrainWarps = 8;
constexpr int kSlab = TBM * TBK * 4;                // bytes of one 128 x 32 slab (16 KB)
constexpr int kStageBytes = 4 * kSlab;              // A hi, A lo, B hi, B lo
constexpr int kEpiRow = 9;                          // float2 per staged row (8 + 1 pad)
constexpr int kEpiWarp = 4096;                      // bytes of one drain warp's staging (4 atoms)
constexpr int kSmemBytes = kStages * kStageBytes + kDrainWarps * kEpiWarp;
constexpr uint64_t kDrainLimitNs = 1000000000ull;   // waits for work already in flight
constexpr int kSpanChunks = 4;                      // k-chunks per drain of the main accumulator

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor (tcgen05) of a K-major operand in the
// 128-byte swizzled layout: start address >> 4, leading byte offset 16 (not
// used by swizzled K-major layouts), stride byte offset 1024 (8-row atoms),
// descriptor version 1, swizzle mode 2 (128 bytes) in bits 61-63.  The atoms
// must start on 1 KB boundaries; a K step inside the 128-byte line advances
// the start address (the hardware applies the swizzle to the full address).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 16, sbo = 1024;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (2ull << 61);
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

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Shared state of one CTA's bounded waits.
struct WaitCtl {
  volatile int* abort;
  int* err;
  uint64_t limit_ns;
};

// Waits for the phase of `bar` with the given parity.  Gives up when another
// thread has aborted, or after limit_ns (then aborts the CTA itself).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const WaitCtl& w) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*w.abort) return false;
    if (globaltimer() - t0 > w.limit_ns) {
      *w.abort = 1;
      atomicExch(w.err, 1);
      return false;
    }
  }
}

// Waits for work already in flight (copies, products) before the CTA exits:
// ignores the abort flag, fixed limit.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if (globaltimer() - t0 > kDrainLimitNs) return false;
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared, completion counted on `bar` (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bulk copy shared -> global (bulk-group completion), and its waits.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Knuth's two-sum: (s, e) with s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int kPasses, int kSpan, bool kPackedOut>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const TcUnit* __restrict__ units, const int32_t* __restrict__ cta_start,
                   const GemmTask* __restrict__ tasks,
                   const TcSeg* __restrict__ segs, const float* __restrict__ Ahi,
                   const float* __restrict__ Alo, const float* __restrict__ Bhi,
                   const float* __restrict__ Blo, float* __restrict__ Chi,
                   float* __restrict__ Clo, int* __restrict__ err, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr bool kLo = kPasses == 3;
  constexpr uint32_t kTmemCols = 512;
  constexpr int kMain = kLo ? 2 : 4;                 // main buffers of 128 columns
  constexpr uint32_t kCorrCol = kMain * TBN;         // two correction buffers (3xTF32)
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ __align__(8) uint64_t mfull[kMain], mempty[kMain], cfull[2], cempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kMain; ++b) {
      mbar_init(&mfull[b], 1);
      mbar_init(&mempty[b], kDrainWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&cfull[b], 1);
      mbar_init(&cempty[b], kDrainWarps);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const WaitCtl wc{&abort_flag, err, wait_ns};
  const int u_begin = cta_start[blockIdx.x], u_end = cta_start[blockIdx.x + 1];
  if (warp < kFirstDrainWarp) asm volatile("setmaxnreg.dec.sync.aligned.u32 56;" ::: "memory");

  if (warp == 0) {
    // ---------------- bulk-copy producer ----------------
    if (lane == 0) {
      int pend[kStages];
#pragma unroll
      for (int s = 0; s < kStages; ++s) pend[s] = -1;
      uint32_t q = 0;
      bool ok = true;
      for (int u = u_begin; u < u_end && ok; ++u) {
        const TcUnit un = units[u];
        const GemmTask t = tasks[un.task];
        for (int k = 0; k < t.nseg && ok; ++k) {
          const TcSeg sg = segs[t.seg0 + k];
          const int ga = min(16, sg.ra8 - un.tm * 16), gb = min(16, sg.rb8 - un.tn * 16);
          const uint32_t ba = (uint32_t)ga * 1024u, bb = (uint32_t)gb * 1024u;
          for (int c = 0; c < sg.kc; ++c, ++q) {
            const int st = (int)(q % kStages);
            if (q >= (uint32_t)kStages && !mbar_wait(&empty[st], ((q / kStages) - 1) & 1, wc)) {
              ok = false;
              break;
            }
            unsigned char* base = smem + st * kStageBytes;
            const int64_t oa = sg.pa + ((int64_t)c * sg.ra8 + un.tm * 16) * kPackTile;
            const int64_t ob = sg.pb + ((int64_t)c * sg.rb8 + un.tn * 16) * kPackTile;
            mbar_expect_tx(&full[st], (ba + bb) * (kLo ? 2u : 1u));
            bulk_g2s(base, Ahi + oa, ba, &full[st]);
            bulk_g2s(base + 2 * kSlab, Bhi + ob, bb, &full[st]);
            if (kLo) {
              bulk_g2s(base + kSlab, Alo + oa, ba, &full[st]);
              bulk_g2s(base + 3 * kSlab, Blo + ob, bb, &full[st]);
            }
            pend[st] = (int)((q / kStages) & 1);
          }
        }
      }
      // copies still in flight must land before the CTA's memory is released
      for (int s = 0; s < kStages; ++s)
        if (pend[s] >= 0) mbar_drain(&full[s], (uint32_t)pend[s]);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t q = 0, p = 0, uc = 0;
      bool ok = true;
      for (int u = u_begin; u < u_end && ok; ++u) {
        const TcUnit un = units[u];
        const int T = un.nchunks;
        if (T == 0) continue;
        // MMA width: the columns of this tile, rounded up to a multiple of 16
        const int nrem = min(TBN, tasks[un.task].N - un.tn * TBN);
        const uint32_t idesc = idesc_tf32(TBM, (nrem + 15) & ~15);
        const uint32_t cb = uc & 1;
        const uint32_t dcorr = tmem + kCorrCol + cb * TBN;
        if (kLo && uc >= 2 && !mbar_wait(&cempty[cb], ((uc >> 1) - 1) & 1, wc)) break;
        uint32_t dmain = 0;
        for (int t = 0; t < T; ++t, ++q) {
          const bool span0 = t % kSpan == 0;
          if (span0) {
            const uint32_t mb = p % kMain;
            if (p >= (uint32_t)kMain && !mbar_wait(&mempty[mb], ((p / kMain) - 1) & 1, wc)) {
              ok = false;
              break;
            }
            dmain = tmem + mb * TBN;
          }
          const int st = (int)(q % kStages);
          if (!mbar_wait(&full[st], (q / kStages) & 1, wc)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* base = smem + st * kStageBytes;
          const uint32_t sah = smem_u32(base), sal = sah + kSlab;
          const uint32_t sbh = sah + 2 * kSlab, sbl = sah + 3 * kSlab;
#pragma unroll
          for (int kk = 0; kk < TBK / 8; ++kk) {     // K = 8 per instruction (32 bytes)
            const uint32_t off = kk * 32;            // 8 k = 32 bytes of the 128-byte line
            mma_tf32(dmain, smem_desc(sah + off), smem_desc(sbh + off), idesc,
                     (span0 && kk == 0) ? 0u : 1u);
            if (kLo) {
              mma_tf32(dcorr, smem_desc(sah + off), smem_desc(sbl + off), idesc,
                       (t == 0 && kk == 0) ? 0u : 1u);
              mma_tf32(dcorr, smem_desc(sal + off), smem_desc(sbh + off), idesc, 1u);
            }
          }
          mma_commit(&empty[st]);                    // the stage is free once these are done
          if (t % kSpan == kSpan - 1 || t == T - 1) {
            mma_commit(&mfull[p % kMain]);           // a span of main products is ready
            ++p;
          }
        }
        if (!ok) break;
        if (kLo) mma_commit(&cfull[cb]);
        ++uc;
      }
      // every product issued must finish before the tensor memory is freed
      mma_commit(&done);
      mbar_drain(&done, 0);
    }
    __syncwarp();
  } else if (warp >= kFirstDrainWarp) {
    // ---------------- drain and epilogue ----------------
    asm volatile("setmaxnreg.inc.sync.aligned.u32 224;" ::: "memory");
    const int quarter = warp & 3, half = (warp - kFirstDrainWarp) >> 2;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t col0 = (uint32_t)(half * 64);
    float2* stage_out =
        reinterpret_cast<float2*>(smem + kStages * kStageBytes + (warp - kFirstDrainWarp) * kEpiWarp);
    uint32_t p = 0, uc = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      const TcUnit un = units[u];
      const GemmTask t = tasks[un.task];
      float ah[64], al[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        ah[j] = 0.f;
        al[j] = 0.f;
      }
      // columns the MMA writes (its width; the rest of the buffer is stale)
      const int nmma = (min(TBN, t.N - un.tn * TBN) + 15) & ~15;
      if (un.nchunks > 0) {
        const int nsp = (un.nchunks + kSpan - 1) / kSpan;
        for (int j = 0; j < nsp; ++j, ++p) {
          const uint32_t mb = p % kMain;
          // one decision per warp: tcgen05.ld is a warp-wide instruction
          if (!__all_sync(0xffffffffu, mbar_wait(&mfull[mb], (p / kMain) & 1, wc))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            if ((int)col0 + h * 16 >= nmma) break;
            uint32_t v[16];
            tmem_ld16(tmem + lane_off + mb * TBN + col0 + h * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              float s, e;
              two_sum(ah[h * 16 + i], __uint_as_float(v[i]), s, e);
              ah[h * 16 + i] = s;
              al[h * 16 + i] = __fadd_rn(al[h * 16 + i], e);
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&mempty[mb]);
        }
        if (!ok) break;
        if (kLo) {
          const uint32_t cb = uc & 1;
          if (!__all_sync(0xffffffffu, mbar_wait(&cfull[cb], (uc >> 1) & 1, wc))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            if ((int)col0 + h * 16 >= nmma) break;
            uint32_t v[16];
            tmem_ld16(tmem + lane_off + kCorrCol + cb * TBN + col0 + h * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i)
              al[h * 16 + i] = __fadd_rn(al[h * 16 + i], __uint_as_float(v[i]));
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&cempty[cb]);
        }
        ++uc;
      }
      const int row0 = un.tm * TBM + quarter * 32;
      const int n0 = un.tn * TBN + half * 64;
      if (kPackedOut) {
        // packed split operand of the next stage: the warp's 32 rows are 4
        // whole 8-row atoms of each 32-wide k-chunk, contiguous in global
        // memory; they are staged in shared memory in the swizzled order
        // (lane = row) and written with one bulk copy per chunk and part
        const int R8 = t.ldc, KC32 = (t.N + 31) / 32 * 32;
        const int g0 = row0 >> 3, ng = min(4, R8 - g0);
        const int r = row0 + lane, rr = lane & 7;
        unsigned char* stg = reinterpret_cast<unsigned char*>(stage_out);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k0 = n0 + 32 * h;
          if (k0 >= KC32 || ng <= 0) break;
#pragma unroll
          for (int part = 0; part < (kLo ? 2 : 1); ++part) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float v[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int kk = 32 * h + 4 * j + i;
                float x = 0.f;
                if (r < t.M && k0 + 4 * j + i < t.N) {
                  const float a = ah[kk], hv = to_tf32(a);
                  // a - hv is exact (hv is a rounded to the 10-bit TF32 mantissa)
                  x = part == 0 ? hv : to_tf32(__fadd_rn(__fsub_rn(a, hv), al[kk]));
                }
                v[i] = x;
              }
              *reinterpret_cast<float4*>(stg + (lane >> 3) * 1024 + rr * 128 + ((j ^ rr) << 4)) =
                  make_float4(v[0], v[1], v[2], v[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              float* dst = (part == 0 ? Chi : Clo) + t.offC + ((int64_t)(k0 >> 5) * R8 + g0) * kPackTile;
              bulk_s2g(dst, stg, (uint32_t)ng * 1024u);
              bulk_wait_read();            // the staging buffer is reused next
            }
            __syncwarp();
          }
        }
      } else {
        // renormalise (hi, lo) and store: 8 columns at a time through the
        // warp's staging rows, written back as rows of 8 consecutive pairs
        float2* C = reinterpret_cast<float2*>(Chi);
#pragma unroll
        for (int c8 = 0; c8 < 64; c8 += 8) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            float s, e;
            two_sum(ah[c8 + i], al[c8 + i], s, e);
            stage_out[lane * kEpiRow + i] = make_float2(s, e);
          }
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int r = it * 4 + (lane >> 3), cc = lane & 7;
            const int gm = row0 + r, gn = n0 + c8 + cc;
            if (gm < t.M && gn < t.N)
              C[t.offC + (int64_t)gm * t.ldc + gn] = stage_out[r * kEpiRow + cc];
          }
          __syncwarp();
        }
      }
    }
    if (kPackedOut && lane == 0) bulk_wait_all();   // the tile stores are complete
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// hi + lo split of a double without FP64 arithmetic (GB300's FP64 pipe would
// bound the packing): hi = x rounded to 11 significant bits (to nearest, ties
// away from zero, from the integer significand), lo = tf32(x - hi) with the
// exact remainder formed from the significand bits.  Returns false for
// values outside the FP32 normal range and for Inf/NaN, which the caller
// splits the plain way.
__device__ __forceinline__ bool split_bits(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const int e = (int)((hw >> 20) & 0x7FF);
  const uint32_t sign = hw & 0x80000000u;
  if (e == 0) {                       // zero or an FP64 subnormal (below the FP32 range)
    hi = __uint_as_float(sign);
    lo = 0.f;
    return true;
  }
  const int ef = e - 1023 + 127;
  if (e == 0x7FF || ef <= 0 || ef >= 254) return false;
  const int hm = (int)((hw & 0xFFFFFu) | 0x100000u);      // top 21 significand bits
  const int r = (hm >> 10) + ((hm >> 9) & 1);              // 11 bits, rounded half away
  hi = __uint_as_float(sign | (((uint32_t)ef << 23) + ((uint32_t)(r - 1024) << 13)));
  const int dh = hm - (r << 10);                           // |dh| <= 512
  // (x - hi) / 2^(e - 1075) = dh 2^32 + lw, rounded once to FP32 by the sum
  const float rem = __fadd_rn(__fmul_rn((float)dh, 4294967296.f), __uint2float_rn(lw));
  const float v = ldexpf(rem, e - 1075);
  lo = to_tf32(sign ? -v : v);
  return true;
}

// Binary search: the block of tile `tile` (blocks in increasing tile0 order).
template <class T>
__device__ __forceinline__ int block_of_tile(const T* __restrict__ b, int n, int tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One warp per 8 x 32 tile: lane l handles row l / 4 and k = 4 j + l % 4 of
// 16-byte chunk j (j = 0..7), stored at its swizzled position.
__global__ void __launch_bounds__(256)
    pack_kernel(const PackBlock* __restrict__ blocks, int nblocks, int ntiles,
                const double* __restrict__ src, float* __restrict__ hi, float* __restrict__ lo) {
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (tile >= ntiles) return;
  const int lane = threadIdx.x & 31;
  const PackBlock b = blocks[block_of_tile(blocks, nblocks, tile)];
  const int local = tile - b.tile0;                  // tile = (c, g) with local = c R8 + g
  const int c = local / b.R8, g = local - c * b.R8;
  const int rr = lane >> 2, r = g * 8 + rr;
  const int64_t out = b.dst + (int64_t)local * kPackTile + rr * 32 + (lane & 3);
  // a power-of-two scale multiplies the FP32 parts exactly; any other one is
  // applied in FP64 before the split
  const bool f64scale = b.scale != 1.0 && b.pow2 == 0.f;
  const float fs = b.pow2 != 0.f ? b.pow2 : 1.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = c * 32 + j * 4 + (lane & 3);
    float h = 0.f, l = 0.f;
    if (r < b.R && k < b.K) {
      double x = b.trans ? src[b.src + (int64_t)k * b.ld + r] : src[b.src + (int64_t)r * b.ld + k];
      if (f64scale) x *= b.scale;
      if (!split_bits(x, h, l)) {
        h = to_tf32((float)x);
        l = to_tf32((float)(x - (double)h));
      }
      h *= fs;
      l *= fs;
    }
    hi[out + ((j ^ rr) << 2)] = h;
    if (lo) lo[out + ((j ^ rr) << 2)] = l;
  }
}

// Double-float accumulation of a coefficient pair times an input pair.
__device__ __forceinline__ void df_acc(float ch, float cl, float2 x, float& ah, float& al) {
  const float p = __fmul_rn(ch, x.x);
  float pe = __fmaf_rn(ch, x.x, -p);
  pe = __fmaf_rn(ch, x.y, pe);
  pe = __fmaf_rn(cl, x.x, pe);
  float s, e;
  two_sum(ah, p, s, e);
  e = __fadd_rn(e, __fadd_rn(al, pe));
  ah = __fadd_rn(s, e);
  al = __fsub_rn(e, __fsub_rn(ah, s));
}

// Stage 2 into the packed operand of stage 3: one warp per 8 x 32 tile of a
// task's packed output; the value is scale * sum_k coef_k in_k in double-float
// arithmetic, then split hi = tf32(v), lo = tf32(v - hi).
__global__ void __launch_bounds__(256)
    combine_pairs_pack_kernel(const PackOut* __restrict__ outs, int ntasks, int ntiles,
                              const CombTask* __restrict__ tasks, const CombTerm* __restrict__ terms,
                              const float2* __restrict__ in, float* __restrict__ out_hi,
                              float* __restrict__ out_lo, float sh, float sl) {
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (tile >= ntiles) return;
  const int lane = threadIdx.x & 31;
  const int ti = block_of_tile(outs, ntasks, tile);
  const PackOut o = outs[ti];
  const CombTask t = tasks[ti];
  const int local = tile - o.tile0;
  const int c = local / o.R8, g = local - c * o.R8;
  const int rr = lane >> 2, r = g * 8 + rr;
  const int R = o.trans ? t.cols : t.rows, K = o.trans ? t.rows : t.cols;
  const int64_t out = o.dst + (int64_t)local * kPackTile + rr * 32 + (lane & 3);
  const bool scaled = sh != 1.f || sl != 0.f;
#pragma unroll 2
  for (int j = 0; j < 8; ++j) {
    const int k = c * 32 + j * 4 + (lane & 3);
    float h = 0.f, l = 0.f;
    if (r < R && k < K) {
      const int row = o.trans ? k : r, col = o.trans ? r : k;
      float ah = 0.f, al = 0.f;
      for (int m = 0; m < t.nt; ++m) {
        const CombTerm tm = terms[t.t0 + m];
        df_acc(tm.chi, tm.clo, in[tm.offIn + (int64_t)row * tm.ldi + col], ah, al);
      }
      if (scaled) {
        const float xh = ah, xl = al;
        ah = 0.f;
        al = 0.f;
        df_acc(sh, sl, make_float2(xh, xl), ah, al);
      }
      h = to_tf32(ah);
      // ah - h is exact (h is ah rounded to the 10-bit TF32 mantissa)
      l = to_tf32(__fadd_rn(__fsub_rn(ah, h), al));
    }
    out_hi[out + ((j ^ rr) << 2)] = h;
    if (out_lo) out_lo[out + ((j ^ rr) << 2)] = l;
  }
}

template <int P, bool kPacked>
void launch_one(const TcUnit* units, const int32_t* cta_start, int ncta, const GemmTask* tasks,
                const TcSeg* segs, const float* Ah, const float* Al, const float* Bh,
                const float* Bl, float* Chi, float* Clo, int* err, uint64_t wait_ns,
                cudaStream_t st) {
  // the shared-memory limit is a per-device attribute of the kernel
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(done.load() & bit)) {
    cudaFuncSetAttribute(gemm_tc_kernel<P, kSpanChunks, kPacked>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (bit) done.fetch_or(bit);
  }
  gemm_tc_kernel<P, kSpanChunks, kPacked><<<ncta, kThreads, kSmemBytes, st>>>(
      units, cta_start, tasks, segs, Ah, Al, Bh, Bl, Chi, Clo, err, wait_ns);
}

}  // namespace

void launch_pack(const PackBlock* blocks, int nblocks, int ntiles, const double* src, float* hi,
                 float* lo, cudaStream_t st) {
  if (ntiles <= 0 || nblocks <= 0) return;
  count_launch();
  pack_kernel<<<(ntiles + 7) / 8, 256, 0, st>>>(blocks, nblocks, ntiles, src, hi, lo);
}

void launch_combine_pairs_pack(const PackOut* outs, int ntasks, int ntiles, const CombTask* tasks,
                               const CombTerm* terms, const float2* in, float* out_hi,
                               float* out_lo, double scale, cudaStream_t st) {
  if (ntiles <= 0 || ntasks <= 0) return;
  count_launch();
  const float sh = (float)scale, sl = (float)(scale - (double)sh);
  combine_pairs_pack_kernel<<<(ntiles + 7) / 8, 256, 0, st>>>(outs, ntasks, ntiles, tasks, terms,
                                                              in, out_hi, out_lo, sh, sl);
}

void launch_gemm_tc(int passes, bool packed, const TcUnit* units, const int32_t* cta_start,
                    int ncta, const GemmTask* tasks, const TcSeg* segs, const float* Ahi,
                    const float* Alo, const float* Bhi, const float* Blo, float* Chi, float* Clo,
                    int* err, uint64_t wait_ns, cudaStream_t st) {
  if (ncta <= 0) return;
  count_launch();
  if (passes == 3) {
    if (packed)
      launch_one<3, true>(units, cta_start, ncta, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, Clo, err,
                          wait_ns, st);
    else
      launch_one<3, false>(units, cta_start, ncta, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, nullptr,
                           err, wait_ns, st);
  } else {
    if (packed)
      launch_one<1, true>(units, cta_start, ncta, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, Clo, err,
                          wait_ns, st);
    else
      launch_one<1, false>(units, cta_start, ncta, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, nullptr,
                           err, wait_ns, st);
  }
}

}  // namespace dmrg3s
