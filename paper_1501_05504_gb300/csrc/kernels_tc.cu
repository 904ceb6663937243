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
// accumulator is drained every kSpan k-chunks (64 k for kSpan = 2) into
// double-float registers with Knuth's two-sum, so FP32 rounding only ever
// sees a short span of main products; a second main buffer takes the next
// span meanwhile.  No FP64 instruction runs in the kernel (GB300's FP64 rate
// is ~1/1000 of its TF32 rate).
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
// Units (output tiles) are assigned round robin over the CTAs, longest first.
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
constexpr int kEpiWarp = 32 * kEpiRow * 8;          // bytes of one drain warp's staging
constexpr int kSmemBytes = kStages * kStageBytes + kDrainWarps * kEpiWarp;
constexpr uint64_t kDrainLimitNs = 1000000000ull;   // waits for work already in flight

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset 128 (K-adjacent core matrices), stride byte offset 1024 (8-row
// groups), all >> 4; descriptor version 1; no swizzle.
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
    gemm_tc_kernel(const TcUnit* __restrict__ units, int nunits, const GemmTask* __restrict__ tasks,
                   const TcSeg* __restrict__ segs, const float* __restrict__ Ahi,
                   const float* __restrict__ Alo, const float* __restrict__ Bhi,
                   const float* __restrict__ Blo, float* __restrict__ Chi,
                   float* __restrict__ Clo, int* __restrict__ err, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr bool kLo = kPasses == 3;
  constexpr uint32_t kTmemCols = kLo ? 512 : 256;   // main x2 (+ corr x2), 128 columns each
  constexpr uint32_t idesc = idesc_tf32(TBM, TBN);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ __align__(8) uint64_t mfull[2], mempty[2], cfull[2], cempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&mfull[b], 1);
      mbar_init(&mempty[b], kDrainWarps);
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
  if (warp < kFirstDrainWarp) asm volatile("setmaxnreg.dec.sync.aligned.u32 56;" ::: "memory");

  if (warp == 0) {
    // ---------------- bulk-copy producer ----------------
    if (lane == 0) {
      int pend[kStages];
#pragma unroll
      for (int s = 0; s < kStages; ++s) pend[s] = -1;
      uint32_t q = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
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
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int T = units[u].nchunks;
        if (T == 0) continue;
        const uint32_t cb = uc & 1;
        const uint32_t dcorr = tmem + 256u + cb * TBN;
        if (kLo && uc >= 2 && !mbar_wait(&cempty[cb], ((uc >> 1) - 1) & 1, wc)) break;
        uint32_t dmain = 0;
        for (int t = 0; t < T; ++t, ++q) {
          const bool span0 = t % kSpan == 0;
          if (span0) {
            const uint32_t mb = p & 1;
            if (p >= 2 && !mbar_wait(&mempty[mb], ((p >> 1) - 1) & 1, wc)) {
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
            const uint32_t off = kk * 256;           // two core matrices along K
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
            mma_commit(&mfull[p & 1]);               // a span of main products is ready
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
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const TcUnit un = units[u];
      const GemmTask t = tasks[un.task];
      float ah[64], al[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        ah[j] = 0.f;
        al[j] = 0.f;
      }
      if (un.nchunks > 0) {
        const int nsp = (un.nchunks + kSpan - 1) / kSpan;
        for (int j = 0; j < nsp; ++j, ++p) {
          const uint32_t mb = p & 1;
          // one decision per warp: tcgen05.ld is a warp-wide instruction
          if (!__all_sync(0xffffffffu, mbar_wait(&mfull[mb], (p >> 1) & 1, wc))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int h = 0; h < 4; ++h) {
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
            uint32_t v[16];
            tmem_ld16(tmem + lane_off + 256u + cb * TBN + col0 + h * 16, v);
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
        // packed split operand of the next stage: the thread's row r and 4
        // consecutive k form one 16-byte run of a core matrix; the 8 rows of
        // a core matrix are neighbouring lanes, so a warp writes 128-byte runs
        const int r = row0 + lane, R8 = t.ldc;
        const int KC32 = (t.N + 31) / 32 * 32;
        if (r < R8 * 8) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int k = n0 + 4 * q;
            if (k >= KC32) break;
            float hv[4], lv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float sh = 0.f, sl = 0.f;
              if (r < t.M && k + i < t.N) {
                float s, e;
                two_sum(ah[4 * q + i], al[4 * q + i], s, e);
                sh = to_tf32(s);
                // s - sh is exact (sh is s rounded to the 10-bit TF32 mantissa)
                sl = to_tf32(__fadd_rn(__fsub_rn(s, sh), e));
              }
              hv[i] = sh;
              lv[i] = sl;
            }
            const int64_t o = t.offC + ((int64_t)(k >> 5) * R8 + (r >> 3)) * kPackTile +
                              ((k & 31) >> 2) * 32 + (r & 7) * 4;
            *reinterpret_cast<float4*>(Chi + o) = make_float4(hv[0], hv[1], hv[2], hv[3]);
            if (kLo) *reinterpret_cast<float4*>(Clo + o) = make_float4(lv[0], lv[1], lv[2], lv[3]);
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
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
// core matrix j (j = 0..7), so each store is a contiguous 128-byte run.
__global__ void __launch_bounds__(256)
    pack_kernel(const PackBlock* __restrict__ blocks, int nblocks, int ntiles,
                const double* __restrict__ src, float* __restrict__ hi, float* __restrict__ lo) {
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (tile >= ntiles) return;
  const int lane = threadIdx.x & 31;
  const PackBlock b = blocks[block_of_tile(blocks, nblocks, tile)];
  const int local = tile - b.tile0;                  // tile = (c, g) with local = c R8 + g
  const int c = local / b.R8, g = local - c * b.R8;
  const int r = g * 8 + (lane >> 2);
  const int64_t out = b.dst + (int64_t)local * kPackTile + lane;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = c * 32 + j * 4 + (lane & 3);
    float h = 0.f, l = 0.f;
    if (r < b.R && k < b.K) {
      const double x =
          b.scale * (b.trans ? src[b.src + (int64_t)k * b.ld + r] : src[b.src + (int64_t)r * b.ld + k]);
      h = to_tf32((float)x);
      l = to_tf32((float)(x - (double)h));
    }
    hi[out + j * 32] = h;
    if (lo) lo[out + j * 32] = l;
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
  const int r = g * 8 + (lane >> 2);
  const int R = o.trans ? t.cols : t.rows, K = o.trans ? t.rows : t.cols;
  const int64_t out = o.dst + (int64_t)local * kPackTile + lane;
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
    out_hi[out + j * 32] = h;
    if (out_lo) out_lo[out + j * 32] = l;
  }
}

template <int P, bool kPacked>
void launch_one(const TcUnit* units, int nunits, const GemmTask* tasks, const TcSeg* segs,
                const float* Ah, const float* Al, const float* Bh, const float* Bl, float* Chi,
                float* Clo, int* err, uint64_t wait_ns, cudaStream_t st) {
  // the shared-memory limit is a per-device attribute of the kernel
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(done.load() & bit)) {
    cudaFuncSetAttribute(gemm_tc_kernel<P, 2, kPacked>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmemBytes);
    if (bit) done.fetch_or(bit);
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 152;
  const int grid = nunits < nsm ? nunits : nsm;
  gemm_tc_kernel<P, 2, kPacked><<<grid, kThreads, kSmemBytes, st>>>(units, nunits, tasks, segs, Ah,
                                                                    Al, Bh, Bl, Chi, Clo, err,
                                                                    wait_ns);
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

void launch_gemm_tc(int passes, bool packed, const TcUnit* units, int nunits,
                    const GemmTask* tasks, const TcSeg* segs, const float* Ahi, const float* Alo,
                    const float* Bhi, const float* Blo, float* Chi, float* Clo, int* err,
                    uint64_t wait_ns, cudaStream_t st) {
  if (nunits <= 0) return;
  count_launch();
  if (passes == 3) {
    if (packed)
      launch_one<3, true>(units, nunits, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, Clo, err, wait_ns, st);
    else
      launch_one<3, false>(units, nunits, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, nullptr, err, wait_ns,
                           st);
  } else {
    if (packed)
      launch_one<1, true>(units, nunits, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, Clo, err, wait_ns, st);
    else
      launch_one<1, false>(units, nunits, tasks, segs, Ahi, Alo, Bhi, Blo, Chi, nullptr, err, wait_ns,
                           st);
  }
}

}  // namespace dmrg3s
