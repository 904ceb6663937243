// FP64 kernels of the block-sparse contraction (CUDA cores).
//
// The grouped GEMM computes every block product of one contraction step of
// the order (((L M) W) R) of Sec. V of arXiv:1501.05504 in one launch: one CTA
// per 64 x 64 output tile, summing all K-segments of its task.  The
// combination kernel applies the MPO step (T2 = sum W T1), which costs
// O(m^2 d^2 w^2) and is bound by memory bandwidth.
#include <atomic>

#include "kernels.hpp"

namespace dmrg3s {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <Trans TA, Trans TB>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(const GemmTile* __restrict__ tiles,
                                                      const GemmTask* __restrict__ tasks,
                                                      const GemmSeg* __restrict__ segs,
                                                      const double* __restrict__ A,
                                                      const double* __restrict__ B,
                                                      double* __restrict__ C) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const GemmTile tile = tiles[blockIdx.x];
  const GemmTask task = tasks[tile.task];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = tile.tm * BM, n0 = tile.tn * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int sgi = 0; sgi < task.nseg; ++sgi) {
    const GemmSeg sg = segs[task.seg0 + sgi];
    const double* Ap = A + sg.offA;
    const double* Bp = B + sg.offB;
    for (int k0 = 0; k0 < sg.K; k0 += BK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int m, k;
        if (TA == Trans::N) {
          k = tid % 16;
          m = tid / 16 + 16 * r;
        } else {
          m = tid % 64;
          k = tid / 64 + 4 * r;
        }
        const int gm = m0 + m, gk = k0 + k;
        double v = 0.0;
        if (gm < task.M && gk < sg.K)
          v = (TA == Trans::N) ? Ap[(int64_t)gm * sg.lda + gk] : Ap[(int64_t)gk * sg.lda + gm];
        As[k][m] = v * sg.scale;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int n, k;
        if (TB == Trans::N) {
          n = tid % 64;
          k = tid / 64 + 4 * r;
        } else {
          k = tid % 16;
          n = tid / 16 + 16 * r;
        }
        const int gn = n0 + n, gk = k0 + k;
        double v = 0.0;
        if (gn < task.N && gk < sg.K)
          v = (TB == Trans::N) ? Bp[(int64_t)gk * sg.ldb + gn] : Bp[(int64_t)gn * sg.ldb + gk];
        Bs[k][n] = v;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= task.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < task.N) C[task.offC + (int64_t)gm * task.ldc + gn] = acc[i][j];
    }
  }
}

__global__ void __launch_bounds__(256) combine_f64_kernel(const CombChunk* __restrict__ chunks,
                                                         const CombTask* __restrict__ tasks,
                                                         const CombTerm* __restrict__ terms,
                                                         const double* __restrict__ in,
                                                         double* __restrict__ out,
                                                         double scale) {
  const CombChunk ch = chunks[blockIdx.x];
  const CombTask t = tasks[ch.task];
  const int n = ch.nrows * t.cols;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int r = ch.row0 + idx / t.cols, c = idx % t.cols;
    double acc = 0.0;
    for (int k = 0; k < t.nt; ++k) {
      const CombTerm tm = terms[t.t0 + k];
      acc = fma(tm.coef, in[tm.offIn + (int64_t)r * tm.ldi + c], acc);
    }
    out[t.offOut + (int64_t)r * t.ldo + c] = scale * acc;
  }
}

// ---- double-float combinations (inputs: tensor-core output pairs) ----
// Knuth's two-sum and an FMA-based product keep ~48 bits; all on the FP32
// pipe (the intrinsics also keep the compiler from contracting the sums).
__device__ __forceinline__ void df_acc(float ch, float cl, float2 x, float& ah, float& al) {
  const float p = __fmul_rn(ch, x.x);
  float pe = __fmaf_rn(ch, x.x, -p);
  pe = __fmaf_rn(ch, x.y, pe);
  pe = __fmaf_rn(cl, x.x, pe);
  const float s = __fadd_rn(ah, p);
  const float bb = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  e = __fadd_rn(e, __fadd_rn(al, pe));
  ah = __fadd_rn(s, e);
  al = __fsub_rn(e, __fsub_rn(ah, s));
}

// sum_k coef_k in_k for output element (r, c) of a chunk's task, as a pair
__device__ __forceinline__ void df_combine(const CombTask& t, const CombTerm* __restrict__ terms,
                                           const float2* __restrict__ in, int r, int c, float sh,
                                           float sl, float& ah, float& al) {
  ah = 0.f;
  al = 0.f;
  for (int k = 0; k < t.nt; ++k) {
    const CombTerm tm = terms[t.t0 + k];
    df_acc(tm.chi, tm.clo, in[tm.offIn + (int64_t)r * tm.ldi + c], ah, al);
  }
  if (sh != 1.f || sl != 0.f) {
    const float h = ah, l = al;
    ah = 0.f;
    al = 0.f;
    df_acc(sh, sl, make_float2(h, l), ah, al);
  }
}

__global__ void __launch_bounds__(256) combine_pairs_f64_kernel(
    const CombChunk* __restrict__ chunks, const CombTask* __restrict__ tasks,
    const CombTerm* __restrict__ terms, const float2* __restrict__ in, double* __restrict__ out,
    float sh, float sl) {
  const CombChunk ch = chunks[blockIdx.x];
  const CombTask t = tasks[ch.task];
  const int n = ch.nrows * t.cols;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int r = ch.row0 + idx / t.cols, c = idx % t.cols;
    float ah, al;
    df_combine(t, terms, in, r, c, sh, sl, ah, al);
    out[t.offOut + (int64_t)r * t.ldo + c] = (double)ah + (double)al;
  }
}

std::atomic<int64_t> g_launches{0};

__global__ void __launch_bounds__(256) dots_kernel(const DotTask* __restrict__ tasks,
                                                   const DotSeg* __restrict__ segs,
                                                   const double* __restrict__ A,
                                                   const double* __restrict__ B,
                                                   double* __restrict__ out) {
  const DotTask t = tasks[blockIdx.x];
  double acc = 0.0;
  for (int k = 0; k < t.nseg; ++k) {
    const DotSeg g = segs[t.seg0 + k];
    for (int64_t e = threadIdx.x; e < g.len; e += blockDim.x)
      acc = fma(A[g.offA + e], B[g.offB + e], acc);
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    out[t.out] = sum;
  }
}

}  // namespace

int64_t launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }

void launch_gemm_f64(Trans ta, Trans tb, const GemmTile* tiles, int ntiles, const GemmTask* tasks,
                     const GemmSeg* segs, const double* A, const double* B, double* C,
                     cudaStream_t st) {
  if (ntiles <= 0) return;
  count_launch();
  dim3 grid(ntiles), block(NT);
  if (ta == Trans::N && tb == Trans::N)
    gemm_f64_kernel<Trans::N, Trans::N><<<grid, block, 0, st>>>(tiles, tasks, segs, A, B, C);
  else if (ta == Trans::N && tb == Trans::T)
    gemm_f64_kernel<Trans::N, Trans::T><<<grid, block, 0, st>>>(tiles, tasks, segs, A, B, C);
  else if (ta == Trans::T && tb == Trans::N)
    gemm_f64_kernel<Trans::T, Trans::N><<<grid, block, 0, st>>>(tiles, tasks, segs, A, B, C);
  else
    gemm_f64_kernel<Trans::T, Trans::T><<<grid, block, 0, st>>>(tiles, tasks, segs, A, B, C);
}

void launch_combine_pairs_f64(const CombChunk* chunks, int nchunks, const CombTask* tasks,
                              const CombTerm* terms, const float2* in, double* out,
                              double scale, cudaStream_t st) {
  if (nchunks <= 0) return;
  count_launch();
  const float sh = (float)scale, sl = (float)(scale - (double)sh);
  combine_pairs_f64_kernel<<<nchunks, 256, 0, st>>>(chunks, tasks, terms, in, out, sh, sl);
}

void launch_combine_f64(const CombChunk* chunks, int nchunks, const CombTask* tasks,
                        const CombTerm* terms, const double* in, double* out, double scale,
                        cudaStream_t st) {
  if (nchunks <= 0) return;
  count_launch();
  combine_f64_kernel<<<nchunks, 256, 0, st>>>(chunks, tasks, terms, in, out, scale);
}

void launch_dots(const DotTask* tasks, int ntasks, const DotSeg* segs, const double* A,
                 const double* B, double* out, cudaStream_t st) {
  if (ntasks <= 0) return;
  count_launch();
  dots_kernel<<<ntasks, 256, 0, st>>>(tasks, segs, A, B, out);
}

}  // namespace dmrg3s
