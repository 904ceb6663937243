// Device task tables and launchers of the block-sparse contraction kernels.
//
// All operand addresses are element offsets relative to base pointers passed
// at launch, so one uploaded table serves every matrix-vector product of a
// Lanczos run (only the vector pointers change).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dmrg3s {

// One K-segment of a grouped GEMM task: C += scale * op(A) op(B) over K.
struct GemmSeg {
  int64_t offA, offB;
  int32_t lda, ldb, K, pad;
  double scale;
};

// One output block C (M x N, row-major with leading dimension ldc) of a
// grouped GEMM.  Segments [seg0, seg0 + nseg) are summed; nseg == 0 writes 0.
struct GemmTask {
  int64_t offC;
  int32_t ldc, M, N, seg0, nseg, pad;
};

// One 64 x 64 output tile of a task.
struct GemmTile {
  int32_t task, tm, tn, pad;
};

// Linear combination of blocks: out = sum_k coef_k in_k (rows x cols).
struct CombTask {
  int64_t offOut;
  int32_t ldo, rows, cols, t0, nt, pad;
};
struct CombTerm {
  int64_t offIn;
  int32_t ldi;
  float chi;        // coef = chi + clo (FP32 pair, filled by the planner)
  double coef;
  float clo;
  int32_t pad;
};
// Work unit of the combination kernel: up to kCombRows rows of one task.
struct CombChunk {
  int32_t task, row0, nrows, pad;
};
constexpr int kCombRows = 16;

enum class Trans { N, T };

// ---- tensor-core operands: packed tiles ----
// A packed matrix (R x K) is stored in tiles of 8 rows x 32 k, tile (g, c) at
// float offset (c * R8 + g) * 256 (R8 = ceil(R / 8) row groups, KC =
// ceil(K / 32) k-chunks).  A tile is one 1 KB atom of the K-major 128-byte
// swizzled layout of the tcgen05 shared-memory descriptors: row r % 8 is a
// 128-byte line (32 k), and its 16-byte chunk j = (k % 32) / 4 sits at chunk
// position j ^ (r % 8), i.e. element (r, k) at float offset (r % 8) * 32 +
// (((k % 32) / 4) ^ (r % 8)) * 4 + k % 4 (the swizzle spreads the eight rows
// the tensor core reads together over all shared-memory banks).  Entries
// beyond R or K are zero.  A 128-row slab of one k-chunk is therefore
// contiguous (16 KB) and moves into shared memory with one bulk copy.  Every
// operand has a hi and a lo part (the 3xTF32 split) at the same offsets of
// two arrays.
constexpr int kPackTile = 256;             // floats per 8 x 32 tile
struct PackBlock {
  // element (r, k) of the packed matrix is scale * src[off + r * ld + k]
  // (trans = 0) or scale * src[off + k * ld + r] (trans = 1)
  int64_t src, dst;                        // dst: float offset of tile (0, 0)
  double scale;
  int32_t ld, R, K, trans, R8, KC, tile0;  // tile0: first tile in the launch numbering
  float pow2;                              // scale when it is a power of two (applied to the
                                           // FP32 parts, exactly), else 0
};
// One K-segment of a tensor-core task: packed A (rows M) and B (rows N).
struct TcSeg {
  int64_t pa, pb;
  int32_t ra8, rb8, kc, pad;
};
// One 128 x 128 output tile: the task's K-segments in order, nchunks k-chunks in all.
struct TcUnit {
  int32_t task, tm, tn, nchunks;
};
// A combination task whose output is written packed (the stage-3 operand).
struct PackOut {
  int64_t dst;
  int32_t R8, KC, trans, tile0;
};

// Blockwise inner products: out[task.out] = sum over the task's segments of
// <A[offA .. offA+len), B[offB .. offB+len)> (FP64, fixed summation order).
struct DotSeg {
  int64_t offA, offB, len;
};
struct DotTask {
  int64_t out;
  int32_t seg0, nseg;
};

// Process-wide count of kernels launched by this library.
int64_t launch_count();
void count_launch(int n = 1);

// FP64 grouped GEMM on the CUDA cores.  opA = A (M x K, lda) or A^T (A stored
// K x M); opB = B (K x N, ldb) or B^T (B stored N x K).
void launch_gemm_f64(Trans ta, Trans tb, const GemmTile* tiles, int ntiles, const GemmTask* tasks,
                     const GemmSeg* segs, const double* A, const double* B, double* C,
                     cudaStream_t st);

// out = scale * sum_k coef_k in_k for every task.
// Tensor-core grouped GEMM (tcgen05): passes = 1 (TF32) or 3 (3xTF32) over
// packed operands (hi, lo parts; lo unused when passes == 1), persistent CTAs
// over the units (a static schedule: one unit list per CTA).  Two output forms:
//  - packed = false: every output element as a double-float pair (hi, lo) at
//    (float2*)Chi + offC + m ldc + n (8 bytes per element, like the double it
//    stands for); Clo unused;
//  - packed = true: the output block packed as the A operand of a following
//    tensor-core stage (R = M rows, K = N, tile layout above, hi at Chi, lo at
//    Clo, lo only with passes == 3), with offC = its float offset and ldc =
//    its R8; entries beyond N in the last k-chunk and rows M .. 8 R8 - 1 are
//    written as zero.
// err is a device flag set to 1 when a wait gave up after wait_ns nanoseconds.
// One CTA per unit list: CTA b runs units [cta_start[b], cta_start[b + 1]).
void launch_gemm_tc(int passes, bool packed, const TcUnit* units, const int32_t* cta_start,
                    int ncta, const GemmTask* tasks, const TcSeg* segs, const float* Ahi,
                    const float* Alo, const float* Bhi, const float* Blo, float* Chi, float* Clo,
                    int* err, uint64_t wait_ns, cudaStream_t st);

// Packs FP64 blocks into tensor-core operands: hi = tf32(x), lo = tf32(x - hi)
// (lo may be null), in the tile layout above.
void launch_pack(const PackBlock* blocks, int nblocks, int ntiles, const double* src, float* hi,
                 float* lo, cudaStream_t st);

// Combinations of double-float pair inputs (the tensor-core outputs), in
// double-float arithmetic on the FP32 pipe: out = scale * sum_k coef_k in_k.
// _pack writes the result as the packed 3xTF32 operand (hi, lo; lo may be
// null) of a following tensor-core stage (one PackOut per task), _f64 writes
// FP64.
void launch_combine_pairs_pack(const PackOut* outs, int ntasks, int ntiles, const CombTask* tasks,
                               const CombTerm* terms, const float2* in, float* out_hi,
                               float* out_lo, double scale, cudaStream_t st);
void launch_combine_pairs_f64(const CombChunk* chunks, int nchunks, const CombTask* tasks,
                              const CombTerm* terms, const float2* in, double* out,
                              double scale, cudaStream_t st);

void launch_combine_f64(const CombChunk* chunks, int nchunks, const CombTask* tasks,
                        const CombTerm* terms, const double* in, double* out, double scale,
                        cudaStream_t st);

// One CTA per task; deterministic (no atomics).
void launch_dots(const DotTask* tasks, int ntasks, const DotSeg* segs, const double* A,
                 const double* B, double* out, cudaStream_t st);

}  // namespace dmrg3s
