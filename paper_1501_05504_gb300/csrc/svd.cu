// FP64 SVD of the truncation step (Sec. IV A, Sec. V step 4): cuSOLVER QR,
// then the one-sided Jacobi method on R^T in this library's kernels.
//
// One-sided Jacobi (Hestenes): plane rotations of column pairs (a, b) of a
// matrix Y, each chosen so that the rotated pair is orthogonal; repeated over
// all pairs until every pair is orthogonal to the tolerance.  For a pair with
// Gram entries alpha = |y_a|^2, beta = |y_b|^2, gamma = <y_a, y_b>, the angle
// has t = tan(theta) the smaller root of t^2 + 2 zeta t - 1 = 0, zeta =
// (beta - alpha) / (2 gamma), and
//   y_a <- c y_a - s y_b,   y_b <- s y_a + c y_b,   c = 1/sqrt(1+t^2), s = c t,
// after which <y_a, y_b> = 0 in exact arithmetic.  A pair is rotated only when
// |gamma| > tol sqrt(alpha beta), tol = max(sqrt(n), 32) 2^-52 (relative
// orthogonality; the floor keeps tol above the rounding error of the computed
// dot product, which would otherwise restart rotations of pairs with equal
// norms indefinitely).
//
// Working on R^T (A P = Q R, Householder QR of A with its columns in
// descending norm order) instead of A: the singular values of a truncated MPS
// span many orders of magnitude, and on such matrices the method needs several
// times fewer sweeps on R^T than on A; the norm order cuts the sweeps on the
// most graded sectors by a further third.
//
// Parallel order: the circle (round-robin) schedule.  With n' = n rounded up
// to even and N = n' - 1, round r (0 <= r < N) pairs column r with N and
// (r + k) mod N with (r - k) mod N for k = 1 .. n'/2 - 1; the N rounds of a
// sweep meet every pair exactly once and the pairs of one round are disjoint
// (a pair with the padding column N = n, n odd, is skipped).  Every pair of a
// round is one CTA and one launch runs a round of every matrix of the batch;
// one sweep (a launch per round) is a CUDA graph.  A matrix with no rotation
// in a sweep is converged and its CTAs exit at once in later sweeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <string>
#include <thread>

#include "kernels.hpp"
#include "svd.hpp"

namespace dmrg3s {

namespace {

constexpr int kJacThreads = 128;

// Device table entry of one matrix.
struct JacJob {
  int64_t offA, offY, offV, offTau;   // Y = R^T (n x n, ld n); V1 (n x n) or offV = -1
  int64_t offS, offVT, offU;          // outputs (offU = -1: no left vectors)
  int32_t m, n, npad, cta0;           // cta0: first CTA of the matrix in a round launch
  int32_t col0;                       // first column of the matrix in the batch numbering
  int32_t nbp, bcta0, pad;            // column blocks (even), first CTA of a block-round launch
};

// Sum of v over the CTA (kJacThreads threads), returned to every thread.
template <class T>
__device__ __forceinline__ T cta_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = red[0];
  for (int w = 1; w < kJacThreads / 32; ++w) s += red[w];
  return s;
}

// Y = R^T from the upper triangle of the factorised A (R[j][i] = A[j + i m],
// j <= i); V1 = I where the left vectors are wanted.  One CTA per column j.
__global__ void __launch_bounds__(kJacThreads)
jac_init_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ col_job,
                const double* __restrict__ A, double* __restrict__ Y, double* __restrict__ V) {
  const JacJob J = jobs[col_job[blockIdx.x]];
  const int j = blockIdx.x - J.col0;
  double* y = Y + J.offY + (int64_t)j * J.n;
  for (int i = threadIdx.x; i < J.n; i += kJacThreads)
    y[i] = i >= j ? A[J.offA + j + (int64_t)i * J.m] : 0.0;
  if (J.offV >= 0) {
    double* v = V + J.offV + (int64_t)j * J.n;
    for (int i = threadIdx.x; i < J.n; i += kJacThreads) v[i] = i == j ? 1.0 : 0.0;
  }
}

// Squared norm of every column of every A (m rows, ld m).  One CTA per column.
__global__ void __launch_bounds__(kJacThreads)
jac_anorm_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ col_job,
                 const double* __restrict__ A, double* __restrict__ nrm) {
  __shared__ double red[kJacThreads / 32];
  const JacJob J = jobs[col_job[blockIdx.x]];
  const int j = blockIdx.x - J.col0;
  const double* x = A + J.offA + (int64_t)j * J.m;
  double s = 0.0;
  for (int i = threadIdx.x; i < J.m; i += kJacThreads) s = fma(x[i], x[i], s);
  s = cta_sum(s, red);
  if (threadIdx.x == 0) nrm[blockIdx.x] = s;
}

// T = A P: column j of T is column perm[j] of A.  One CTA per column.
__global__ void __launch_bounds__(kJacThreads)
jac_permute_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ col_job,
                   const int* __restrict__ perm, const double* __restrict__ A,
                   double* __restrict__ T) {
  const JacJob J = jobs[col_job[blockIdx.x]];
  const int j = blockIdx.x - J.col0;
  const double* x = A + J.offA + (int64_t)perm[blockIdx.x] * J.m;
  double* t = T + J.offA + (int64_t)j * J.m;
  for (int i = threadIdx.x; i < J.m; i += kJacThreads) t[i] = x[i];
}

// Advances the sweep counter read by the round kernels (first node of a sweep).
__global__ void jac_next_sweep_kernel(int* sweep) { *sweep += 1; }

// One round r of the current sweep for every matrix: one CTA per pair.
// rot[s * njobs + job] counts the rotations of sweep s.  The first kJacCache
// elements of each thread's share stay in registers between the dot products
// and the rotation; the rotation itself (a few FP64 divisions and square
// roots) is computed once, by thread 0.
constexpr int kJacCache = 4;
__global__ void __launch_bounds__(kJacThreads)
jac_round_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ cta_job, int njobs, int r,
                 const int* __restrict__ sweep, int* __restrict__ rot, double* __restrict__ Y,
                 double* __restrict__ V) {
  __shared__ double red[3][kJacThreads / 32];
  __shared__ double cs_sn[2];
  __shared__ int go;
  const int sw = *sweep;
  if (sw < 0 || sw >= kJacobiMaxSweeps) return;
  const int jb = cta_job[blockIdx.x];
  if (sw > 0 && rot[(sw - 1) * njobs + jb] == 0) return;   // converged in the previous sweep
  const JacJob J = jobs[jb];
  const int N = J.npad - 1;
  if (r >= N) return;
  const int k = blockIdx.x - J.cta0;
  int a, b;
  if (k == 0) {
    a = r;
    b = N;
  } else {
    a = (r + k) % N;
    b = (r - k + N) % N;
  }
  const int n = J.n;
  if (a >= n || b >= n) return;   // the padding column
  double* ya = Y + J.offY + (int64_t)a * n;
  double* yb = Y + J.offY + (int64_t)b * n;
  double ua[kJacCache], ub[kJacCache];
  double saa = 0.0, sbb = 0.0, sab = 0.0;
#pragma unroll
  for (int e = 0; e < kJacCache; ++e) {
    const int i = threadIdx.x + e * kJacThreads;
    ua[e] = i < n ? ya[i] : 0.0;
    ub[e] = i < n ? yb[i] : 0.0;
    saa = fma(ua[e], ua[e], saa);
    sbb = fma(ub[e], ub[e], sbb);
    sab = fma(ua[e], ub[e], sab);
  }
  for (int i = threadIdx.x + kJacCache * kJacThreads; i < n; i += kJacThreads) {
    const double u = ya[i], v = yb[i];
    saa = fma(u, u, saa);
    sbb = fma(v, v, sbb);
    sab = fma(u, v, sab);
  }
  for (int o = 16; o > 0; o >>= 1) {
    saa += __shfl_xor_sync(0xffffffffu, saa, o);
    sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
    sab += __shfl_xor_sync(0xffffffffu, sab, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = saa;
    red[1][threadIdx.x >> 5] = sbb;
    red[2][threadIdx.x >> 5] = sab;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    saa = red[0][0];
    sbb = red[1][0];
    sab = red[2][0];
    for (int w = 1; w < kJacThreads / 32; ++w) {
      saa += red[0][w];
      sbb += red[1][w];
      sab += red[2][w];
    }
    int g = 0;
    // zero columns and NaN leave the pair unrotated (NaN reaches the singular values)
    if (saa > 0.0 && sbb > 0.0) {
      const double tol = fmax(sqrt((double)n), 32.0) * DBL_EPSILON;
      if (fabs(sab) > tol * sqrt(saa) * sqrt(sbb)) {
        const double zeta = (sbb - saa) / (2.0 * sab);
        const double az = fabs(zeta);
        const double t =
            az > 1e150 ? 0.5 / zeta : copysign(1.0, zeta) / (az + sqrt(1.0 + az * az));
        const double c = 1.0 / sqrt(1.0 + t * t);
        cs_sn[0] = c;
        cs_sn[1] = c * t;
        g = 1;
        atomicAdd(rot + sw * njobs + jb, 1);
      }
    }
    go = g;
  }
  __syncthreads();
  if (!go) return;
  const double cs = cs_sn[0], sn = cs_sn[1];
#pragma unroll
  for (int e = 0; e < kJacCache; ++e) {
    const int i = threadIdx.x + e * kJacThreads;
    if (i < n) {
      ya[i] = cs * ua[e] - sn * ub[e];
      yb[i] = sn * ua[e] + cs * ub[e];
    }
  }
  for (int i = threadIdx.x + kJacCache * kJacThreads; i < n; i += kJacThreads) {
    const double u = ya[i], v = yb[i];
    ya[i] = cs * u - sn * v;
    yb[i] = sn * u + cs * v;
  }
  if (J.offV >= 0) {
    double* va = V + J.offV + (int64_t)a * n;
    double* vb = V + J.offV + (int64_t)b * n;
    for (int i = threadIdx.x; i < n; i += kJacThreads) {
      const double u = va[i], v = vb[i];
      va[i] = cs * u - sn * v;
      vb[i] = sn * u + cs * v;
    }
  }
}

// Block form of a round.  The columns of Y are taken in blocks of KB (nbp
// blocks, an even count, the last ones partly or wholly padding); round r of
// the circle schedule over blocks pairs block r with nbp - 1 and (r + k) mod
// (nbp - 1) with (r - k) mod (nbp - 1), one CTA per block pair.  The CTA
// holds its 2 KB columns in shared memory and runs one cyclic sweep over all
// their pairs (the circle schedule over the 2 KB columns: 2 KB - 1 inner
// rounds, one pair per warp), with the test and rotation of the scalar round;
// then writes them back and applies the same rotations, in the same order,
// to the columns of V1.  A sweep of nbp - 1 block rounds meets every column
// pair at least once, so it is a valid cyclic sweep; the pairs inside a block
// are visited once per block round.  Padding columns are zero and never rotate.
template <int KB>
__global__ void __launch_bounds__(KB * 32)
jac_block_round_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ cta_job,
                       int njobs, int r, const int* __restrict__ sweep, int* __restrict__ rot,
                       double* __restrict__ Y, double* __restrict__ V) {
  extern __shared__ double sm[];
  constexpr int M = 2 * KB;
  const int sw = *sweep;
  if (sw < 0 || sw >= kJacobiMaxSweeps) return;
  const int jb = cta_job[blockIdx.x];
  if (sw > 0 && rot[(sw - 1) * njobs + jb] == 0) return;   // converged in the previous sweep
  const JacJob J = jobs[jb];
  const int N = J.nbp - 1;
  if (r >= N) return;
  const int k = blockIdx.x - J.bcta0;
  int ba, bb;
  if (k == 0) {
    ba = r;
    bb = N;
  } else {
    ba = (r + k) % N;
    bb = (r - k + N) % N;
  }
  const int n = J.n;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double* cols = sm;                                 // M columns of n
  double2* logr = reinterpret_cast<double2*>(sm + (int64_t)M * n);   // (c, s) per inner pair
  auto gcol = [&](int l) { return l < KB ? ba * KB + l : bb * KB + (l - KB); };
  for (int l = 0; l < M; ++l) {
    const int g = gcol(l);
    const double* src = Y + J.offY + (int64_t)g * n;
    for (int i = tid; i < n; i += KB * 32) cols[l * n + i] = g < n ? src[i] : 0.0;
  }
  __syncthreads();
  const double tol = fmax(sqrt((double)n), 32.0) * DBL_EPSILON;
  int nrot = 0;
  for (int ir = 0; ir < M - 1; ++ir) {
    int a, b;
    if (w == 0) {
      a = ir;
      b = M - 1;
    } else {
      a = (ir + w) % (M - 1);
      b = (ir - w + M - 1) % (M - 1);
    }
    double* ya = cols + a * n;
    double* yb = cols + b * n;
    double saa = 0.0, sbb = 0.0, sab = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double u = ya[i], v = yb[i];
      saa = fma(u, u, saa);
      sbb = fma(v, v, sbb);
      sab = fma(u, v, sab);
    }
    for (int o = 16; o > 0; o >>= 1) {
      saa += __shfl_xor_sync(0xffffffffu, saa, o);
      sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
      sab += __shfl_xor_sync(0xffffffffu, sab, o);
    }
    double cs = 1.0, sn = 0.0;
    // zero columns (padding) and NaN leave the pair unrotated
    if (saa > 0.0 && sbb > 0.0 && fabs(sab) > tol * sqrt(saa) * sqrt(sbb)) {
      const double zeta = (sbb - saa) / (2.0 * sab);
      const double az = fabs(zeta);
      const double t =
          az > 1e150 ? 0.5 / zeta : copysign(1.0, zeta) / (az + sqrt(1.0 + az * az));
      cs = 1.0 / sqrt(1.0 + t * t);
      sn = cs * t;
      ++nrot;
      for (int i = lane; i < n; i += 32) {
        const double u = ya[i], v = yb[i];
        ya[i] = cs * u - sn * v;
        yb[i] = sn * u + cs * v;
      }
    }
    if (lane == 0) logr[ir * KB + w] = make_double2(cs, sn);
    __syncthreads();
  }
  for (int l = 0; l < M; ++l) {
    const int g = gcol(l);
    if (g >= n) continue;
    double* dst = Y + J.offY + (int64_t)g * n;
    for (int i = tid; i < n; i += KB * 32) dst[i] = cols[l * n + i];
  }
  if (lane == 0 && nrot > 0) atomicAdd(rot + sw * njobs + jb, nrot);
  if (J.offV < 0) return;
  __syncthreads();
  for (int l = 0; l < M; ++l) {
    const int g = gcol(l);
    const double* src = V + J.offV + (int64_t)g * n;
    for (int i = tid; i < n; i += KB * 32) cols[l * n + i] = g < n ? src[i] : 0.0;
  }
  __syncthreads();
  for (int ir = 0; ir < M - 1; ++ir) {
    int a, b;
    if (w == 0) {
      a = ir;
      b = M - 1;
    } else {
      a = (ir + w) % (M - 1);
      b = (ir - w + M - 1) % (M - 1);
    }
    const double2 r2 = logr[ir * KB + w];
    if (r2.y != 0.0) {
      double* va = cols + a * n;
      double* vb = cols + b * n;
      for (int i = lane; i < n; i += 32) {
        const double u = va[i], v = vb[i];
        va[i] = r2.x * u - r2.y * v;
        vb[i] = r2.y * u + r2.x * v;
      }
    }
    __syncthreads();
  }
  for (int l = 0; l < M; ++l) {
    const int g = gcol(l);
    if (g >= n) continue;
    double* dst = V + J.offV + (int64_t)g * n;
    for (int i = tid; i < n; i += KB * 32) dst[i] = cols[l * n + i];
  }
}

// Shared memory of a block round with KB-column blocks on columns of n.
inline size_t jac_block_smem(int kb, int n) {
  return ((size_t)2 * kb * n + (size_t)(2 * kb - 1) * kb * 2) * sizeof(double);
}
constexpr size_t kJacBlockSmemMax = 200 * 1024;

// sigma of every column of every Y.  One CTA per column.
__global__ void __launch_bounds__(kJacThreads)
jac_norm_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ col_job,
                const double* __restrict__ Y, double* __restrict__ sig) {
  __shared__ double red[kJacThreads / 32];
  const JacJob J = jobs[col_job[blockIdx.x]];
  const int j = blockIdx.x - J.col0;
  const double* y = Y + J.offY + (int64_t)j * J.n;
  double s = 0.0;
  for (int i = threadIdx.x; i < J.n; i += kJacThreads) s = fma(y[i], y[i], s);
  s = cta_sum(s, red);
  if (threadIdx.x == 0) sig[blockIdx.x] = sqrt(s);
}

// Sort key: NaN above everything, so that it lands in S and is seen.
__device__ __forceinline__ double sig_key(double x) { return x != x ? INFINITY : x; }

// Column j of matrix J goes to position c = its rank (descending sigma, ties
// by index): S[c] = sigma_j, VT row c = P y_j / sigma_j (P: the column order
// of the factorised A P), and, when wanted, U column c = (V1 column j; 0),
// which Q then multiplies.  One CTA per column.
__global__ void __launch_bounds__(kJacThreads)
jac_scatter_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ col_job,
                   const int* __restrict__ perm, const double* __restrict__ Y,
                   const double* __restrict__ V, const double* __restrict__ sig,
                   double* __restrict__ S, double* __restrict__ VT, double* __restrict__ U) {
  __shared__ int red[kJacThreads / 32];
  const JacJob J = jobs[col_job[blockIdx.x]];
  const int j = blockIdx.x - J.col0;
  const int n = J.n;
  const double s = sig[blockIdx.x];
  const double ks = sig_key(s);
  int cnt = 0;
  for (int i = threadIdx.x; i < n; i += kJacThreads) {
    const double o = sig_key(sig[J.col0 + i]);
    cnt += (o > ks || (o == ks && i < j)) ? 1 : 0;
  }
  const int c = cta_sum(cnt, red);
  if (threadIdx.x == 0) S[J.offS + c] = s;
  const double* y = Y + J.offY + (int64_t)j * n;
  const int* pj = perm + J.col0;   // row i of R belongs to column pj[i] of A
  for (int i = threadIdx.x; i < n; i += kJacThreads)
    VT[J.offVT + c + (int64_t)pj[i] * n] = s > 0.0 ? y[i] / s : 0.0;
  if (J.offU >= 0) {
    const double* v = V + J.offV + (int64_t)j * n;
    double* u = U + J.offU + (int64_t)c * J.m;
    for (int i = threadIdx.x; i < J.m; i += kJacThreads) u[i] = i < n ? v[i] : 0.0;
  }
}

dmrg3s_status cuda_ok(Context* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DMRG3S_OK;
  return fail(c, DMRG3S_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Dynamic shared memory of the block rounds (above the 48 KB default).
dmrg3s_status jac_block_prepare(Context* c, int kb, size_t smem) {
  cudaError_t e = cudaSuccess;
  if (kb == 16)
    e = cudaFuncSetAttribute(jac_block_round_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  else if (kb == 8)
    e = cudaFuncSetAttribute(jac_block_round_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  else if (kb == 4)
    e = cudaFuncSetAttribute(jac_block_round_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  return cuda_ok(c, e, "Jacobi block rounds");
}

}  // namespace

dmrg3s_status lane_create(Context* c, SvdLane* w) {
  if (cusolverDnCreate(&w->h) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&w->p) != CUSOLVER_STATUS_SUCCESS ||
      cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, DMRG3S_ERR_CUDA, "SVD lane set-up");
  return DMRG3S_OK;
}

void lane_destroy(SvdLane* w) {
  if (w->dwork) cudaFree(w->dwork);
  if (w->p) cusolverDnDestroyParams(w->p);
  if (w->h) cusolverDnDestroy(w->h);
  if (w->ev) cudaEventDestroy(w->ev);
  if (w->s) cudaStreamDestroy(w->s);
  *w = SvdLane();
}

int jacobi_max_sweeps() {
  const char* e = std::getenv("DMRG3S_JACOBI_SWEEPS");
  if (!e) return kJacobiMaxSweeps;
  const int v = std::atoi(e);
  return v < 1 ? 1 : (v > kJacobiMaxSweeps ? kJacobiMaxSweeps : v);
}

dmrg3s_status svd_jacobi(Context* c, std::vector<SvdLane>& lanes, int nlanes,
                         const std::vector<SvdJob>& jobs, double* A, double* S, double* VT,
                         double* U, int* info, cudaStream_t st, std::string* diag,
                         int* sweeps) {
  const int nj = (int)jobs.size();
  if (nj == 0) return DMRG3S_OK;
  if (nlanes < 1 || nlanes > (int)lanes.size()) nlanes = (int)lanes.size();
  if (nlanes < 1) return fail(c, DMRG3S_ERR_ARG, "no SVD lane");
  // ---- tables
  std::vector<JacJob> tab(nj);
  std::vector<int> cta_job, col_job;
  int64_t ny = 0, nv = 0, ntau = 0;
  int maxr = 0;
  for (int k = 0; k < nj; ++k) {
    const SvdJob& jb = jobs[k];
    if (jb.n < 1 || jb.m < jb.n || jb.m > (1 << 30) || jb.n > (1 << 15))
      return fail(c, DMRG3S_ERR_ARG, "SVD matrix shape (need 1 <= n <= m, n <= 32768)");
    if (jb.offU >= 0 && !U) return fail(c, DMRG3S_ERR_ARG, "SVD left vectors without a buffer");
    JacJob& t = tab[k];
    t.offA = jb.offA;
    t.offY = ny;
    ny += jb.n * jb.n;
    t.offV = jb.offU >= 0 ? nv : -1;
    if (jb.offU >= 0) nv += jb.n * jb.n;
    t.offTau = ntau;
    ntau += jb.n;
    t.offS = jb.offS;
    t.offVT = jb.offVT;
    t.offU = jb.offU;
    t.m = (int32_t)jb.m;
    t.n = (int32_t)jb.n;
    t.npad = t.n + (t.n & 1);
    t.cta0 = (int32_t)cta_job.size();
    t.col0 = (int32_t)col_job.size();
    t.pad = 0;
    cta_job.insert(cta_job.end(), t.npad / 2, k);
    col_job.insert(col_job.end(), t.n, k);
    maxr = std::max(maxr, t.npad - 1);
  }
  // block rounds (jac_block_round_kernel) when the widest matrix's 2 KB
  // columns fit in shared memory, with the widest such blocks up to 16
  int nmax = 0;
  for (const JacJob& t : tab) nmax = std::max(nmax, (int)t.n);
  int kb = 0;
  for (int cand : {16, 8, 4})
    if (!kb && jac_block_smem(cand, nmax) <= kJacBlockSmemMax) kb = cand;
  std::vector<int> bcta_job;
  int maxrb = 0;
  if (kb) {
    for (int k = 0; k < nj; ++k) {
      JacJob& t = tab[k];
      const int nb = (t.n + kb - 1) / kb;
      t.nbp = nb + (nb & 1);
      t.bcta0 = (int32_t)bcta_job.size();
      bcta_job.insert(bcta_job.end(), t.nbp / 2, k);
      maxrb = std::max(maxrb, t.nbp - 1);
    }
  }
  const int nbcta = (int)bcta_job.size();
  const int ncta = (int)cta_job.size(), ncol = (int)col_job.size();
  int64_t na = 0;   // extent of the A buffer used by the jobs
  for (const JacJob& t : tab) na = std::max(na, t.offA + (int64_t)t.m * t.n);
  // ---- device buffers: doubles [tau | Y | V1 | sigma | column norms | T = A P],
  //      ints [cta_job | col_job | perm | rot | sweep | qinfo]
  const int64_t nd = ntau + ny + nv + 2 * (int64_t)ncol + na;
  const int64_t ni = ncta + 2 * (int64_t)ncol + (int64_t)kJacobiMaxSweeps * nj + 1 + nj + nbcta;
  double* dd = nullptr;
  int* di = nullptr;
  JacJob* dt = nullptr;
  dmrg3s_status s = DMRG3S_OK;
  if ((s = cuda_ok(c, cudaMallocAsync((void**)&dd, (size_t)nd * sizeof(double), st), "SVD buffers")) ||
      (s = cuda_ok(c, cudaMallocAsync((void**)&di, (size_t)ni * sizeof(int), st), "SVD buffers")) ||
      (s = cuda_ok(c, cudaMallocAsync((void**)&dt, tab.size() * sizeof(JacJob), st), "SVD buffers"))) {
    if (dd) cudaFreeAsync(dd, st);
    if (di) cudaFreeAsync(di, st);
    return s;
  }
  double* tau = dd;
  double* Y = tau + ntau;
  double* V1 = Y + ny;
  double* sig = V1 + nv;
  double* anrm = sig + ncol;
  double* T = anrm + ncol;
  int* d_cta = di;
  int* d_col = d_cta + ncta;
  int* d_perm = d_col + ncol;
  int* rot = d_perm + ncol;
  int* d_sweep = rot + (int64_t)kJacobiMaxSweeps * nj;
  int* qinfo = d_sweep + 1;
  int* d_bcta = qinfo + nj;
  cudaMemcpyAsync(dt, tab.data(), tab.size() * sizeof(JacJob), cudaMemcpyHostToDevice, st);
  if (nbcta)
    cudaMemcpyAsync(d_bcta, bcta_job.data(), bcta_job.size() * sizeof(int), cudaMemcpyHostToDevice,
                    st);
  cudaMemcpyAsync(d_cta, cta_job.data(), cta_job.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_col, col_job.data(), col_job.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(rot, 0, (size_t)kJacobiMaxSweeps * nj * sizeof(int), st);
  cudaMemsetAsync(d_sweep, 0xff, sizeof(int), st);   // -1: the first sweep advances it to 0
  s = cuda_ok(c, cudaGetLastError(), "SVD tables");
  // ---- columns in descending norm order, T = A P: the Jacobi sweeps on R^T
  // of A P need fewer sweeps than on R^T of A when the column norms are graded
  std::vector<int> perm(ncol);
  if (!s) {
    std::vector<double> hn(ncol);
    jac_anorm_kernel<<<ncol, kJacThreads, 0, st>>>(dt, d_col, A, anrm);
    count_launch();
    if (!(s = cuda_ok(c, cudaMemcpyAsync(hn.data(), anrm, ncol * sizeof(double),
                                         cudaMemcpyDeviceToHost, st), "column norms")) &&
        !(s = cuda_ok(c, cudaStreamSynchronize(st), "column norms"))) {
      for (const JacJob& t : tab) {
        int* pj = perm.data() + t.col0;
        for (int i = 0; i < t.n; ++i) pj[i] = i;
        const double* nj_ = hn.data() + t.col0;
        std::stable_sort(pj, pj + t.n, [&](int x, int y) { return nj_[x] > nj_[y]; });
      }
      cudaMemcpyAsync(d_perm, perm.data(), ncol * sizeof(int), cudaMemcpyHostToDevice, st);
      jac_permute_kernel<<<ncol, kJacThreads, 0, st>>>(dt, d_col, d_perm, A, T);
      count_launch();
      s = cuda_ok(c, cudaGetLastError(), "column order");
    }
  }
  // ---- lane workspaces (QR, and Q V1 for the left vectors)
  size_t dmax = 1, hmax = 1;
  for (const JacJob& t : tab) {
    if (s) break;
    size_t wd = 0, wh = 0;
    if (cusolverDnXgeqrf_bufferSize(lanes[0].h, lanes[0].p, t.m, t.n, CUDA_R_64F, T + t.offA, t.m,
                                    CUDA_R_64F, tau + t.offTau, CUDA_R_64F, &wd,
                                    &wh) != CUSOLVER_STATUS_SUCCESS)
      s = fail(c, DMRG3S_ERR_CUDA, "QR buffer size");
    dmax = std::max(dmax, wd);
    hmax = std::max(hmax, wh);
    if (!s && t.offU >= 0) {
      int lw = 0;
      if (cusolverDnDormqr_bufferSize(lanes[0].h, CUBLAS_SIDE_LEFT, CUBLAS_OP_N, t.m, t.n, t.n,
                                      T + t.offA, t.m, tau + t.offTau, U + t.offU, t.m,
                                      &lw) != CUSOLVER_STATUS_SUCCESS)
        s = fail(c, DMRG3S_ERR_CUDA, "ormqr buffer size");
      dmax = std::max(dmax, (size_t)lw * sizeof(double));
    }
  }
  for (int w = 0; !s && w < nlanes; ++w) {
    SvdLane& l = lanes[w];
    if (l.dbytes < dmax) {
      if (l.dwork) cudaFree(l.dwork);
      l.dwork = nullptr;
      l.dbytes = 0;
      if (cudaMalloc(&l.dwork, dmax) != cudaSuccess) {
        s = fail(c, DMRG3S_ERR_CUDA, "SVD workspace");
        break;
      }
      l.dbytes = dmax;
    }
    if (l.hwork.size() < hmax) l.hwork.resize(hmax);
  }
  // greedy assignment to lanes by QR cost m n^2, largest first
  std::vector<int> order(nj);
  for (int k = 0; k < nj; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)tab[a].m * tab[a].n * tab[a].n > (double)tab[b].m * tab[b].n * tab[b].n;
  });
  std::vector<std::vector<int>> part(nlanes);
  std::vector<double> load(nlanes, 0.0);
  for (int k : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    part[w].push_back(k);
    load[w] += (double)tab[k].m * tab[k].n * tab[k].n + 1e5;
  }
  cudaEvent_t ev_in = nullptr;
  if (!s && cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) != cudaSuccess)
    s = fail(c, DMRG3S_ERR_CUDA, "SVD event");
  // runs fn(lane, job) for every wanted job on its lane after the work queued
  // on st; st waits for the lanes
  auto on_lanes = [&](auto fn, auto wanted) -> bool {
    cudaEventRecord(ev_in, st);
    std::vector<int> bad(nlanes, 0);
    auto run = [&](int w) {
      SvdLane& l = lanes[w];
      cudaSetDevice(c->device);
      cudaStreamWaitEvent(l.s, ev_in, 0);
      cusolverDnSetStream(l.h, l.s);
      for (int k : part[w])
        if (wanted(k) && !fn(l, k)) bad[w] = 1;
      cudaEventRecord(l.ev, l.s);
    };
    std::vector<std::thread> th;
    for (int w = 1; w < nlanes; ++w)
      if (!part[w].empty()) th.emplace_back(run, w);
    if (!part[0].empty()) run(0);
    for (auto& t : th) t.join();
    bool ok = true;
    for (int w = 0; w < nlanes; ++w) {
      ok = ok && !bad[w];
      if (!part[w].empty()) cudaStreamWaitEvent(st, lanes[w].ev, 0);
    }
    return ok;
  };
  auto all = [](int) { return true; };
  // ---- 1. A = Q R
  const bool qr_ok = s || on_lanes(
      [&](SvdLane& l, int k) {
        const JacJob& t = tab[k];
        return cusolverDnXgeqrf(l.h, l.p, t.m, t.n, CUDA_R_64F, T + t.offA, t.m, CUDA_R_64F,
                                tau + t.offTau, CUDA_R_64F, l.dwork, l.dbytes, l.hwork.data(),
                                l.hwork.size(), qinfo + k) == CUSOLVER_STATUS_SUCCESS;
      },
      all);
  if (!s && !qr_ok) s = fail(c, DMRG3S_ERR_CUDA, "QR factorisation");
  // ---- 2. Y = R^T, V1 = I
  if (!s) {
    jac_init_kernel<<<ncol, kJacThreads, 0, st>>>(dt, d_col, T, Y, V1);
    count_launch();
    s = cuda_ok(c, cudaGetLastError(), "Jacobi set-up");
  }
  // ---- 3. sweeps: one CUDA graph of (sweep counter, rounds 0 .. maxr-1),
  // block rounds where they fit
  const size_t bsmem = kb ? jac_block_smem(kb, nmax) : 0;
  if (!s && kb && (s = jac_block_prepare(c, kb, bsmem))) kb = 0;
  const int nround = kb ? maxrb : maxr;
  auto enqueue_sweep = [&](cudaStream_t q) {
    jac_next_sweep_kernel<<<1, 1, 0, q>>>(d_sweep);
    for (int r = 0; r < nround; ++r) {
      if (kb == 16)
        jac_block_round_kernel<16><<<nbcta, 16 * 32, bsmem, q>>>(dt, d_bcta, nj, r, d_sweep, rot, Y, V1);
      else if (kb == 8)
        jac_block_round_kernel<8><<<nbcta, 8 * 32, bsmem, q>>>(dt, d_bcta, nj, r, d_sweep, rot, Y, V1);
      else if (kb == 4)
        jac_block_round_kernel<4><<<nbcta, 4 * 32, bsmem, q>>>(dt, d_bcta, nj, r, d_sweep, rot, Y, V1);
      else
        jac_round_kernel<<<ncta, kJacThreads, 0, q>>>(dt, d_cta, nj, r, d_sweep, rot, Y, V1);
    }
  };
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  if (!s && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
      cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    enqueue_sweep(cap);
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess ||
        cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess)
      gexec = nullptr;
  }
  cudaGetLastError();   // a failed capture leaves the plain launches below
  std::vector<int> hrot(nj), active(nj, 1);
  std::vector<int> conv(nj, 0);
  Profiler& pr = c->prof;
  const int max_sweeps = jacobi_max_sweeps();
  if (sweeps) *sweeps = 0;
  for (int sw = 0; !s && sw < max_sweeps; ++sw) {
    if (sweeps) *sweeps = sw + 1;
    const int id = pr.on ? pr.begin(kProfJacobi, 0.0, 0.0, st) : -1;
    if (gexec) {
      s = cuda_ok(c, cudaGraphLaunch(gexec, st), "Jacobi sweep");
    } else {
      enqueue_sweep(st);
      s = cuda_ok(c, cudaGetLastError(), "Jacobi sweep");
    }
    count_launch(nround + 1);
    if (id >= 0) pr.end(id, st);
    if (s) break;
    if ((s = cuda_ok(c, cudaMemcpyAsync(hrot.data(), rot + (int64_t)sw * nj, nj * sizeof(int),
                                        cudaMemcpyDeviceToHost, st), "Jacobi rotations")) ||
        (s = cuda_ok(c, cudaStreamSynchronize(st), "Jacobi sweep")))
      break;
    // cost of the sweep: a pair test reads two columns (16n bytes) for three
    // dot products (6n flops); a rotation of a column pair of Y and of V1
    // takes 6n flops each and writes 16n bytes each (V1 also read).  Block
    // rounds test every pair of their 2 kb columns, from shared memory, and
    // move each column between memory and the CTA twice (Y, and V1).
    double fl = 0.0, by = 0.0;
    bool more = false;
    for (int k = 0; k < nj; ++k) {
      if (!active[k]) continue;
      const double n = tab[k].n;
      const bool v = tab[k].offV >= 0;
      if (kb) {
        const double ctas = (tab[k].nbp - 1.0) * (tab[k].nbp / 2), m2 = 2.0 * kb;
        fl += ctas * 0.5 * m2 * (m2 - 1.0) * 6.0 * n + hrot[k] * 6.0 * n * (v ? 2.0 : 1.0);
        by += ctas * m2 * 16.0 * n * (v ? 2.0 : 1.0);
      } else {
        const double pairs = 0.5 * n * (n - 1.0);
        fl += pairs * 6.0 * n + hrot[k] * 6.0 * n * (v ? 2.0 : 1.0);
        by += pairs * 16.0 * n + hrot[k] * 16.0 * n * (v ? 3.0 : 1.0);
      }
      if (hrot[k] == 0) {
        active[k] = 0;
        conv[k] = 1;
      } else {
        more = true;
      }
    }
    if (id >= 0) {
      pr.recs[id].flops = fl;
      pr.recs[id].bytes = by;
      pr.recs[id].launches = nround + 1;
    }
    if (!more) break;
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  // ---- 4. singular values in descending order, VT, (V1; 0) for the left vectors
  if (!s) {
    jac_norm_kernel<<<ncol, kJacThreads, 0, st>>>(dt, d_col, Y, sig);
    jac_scatter_kernel<<<ncol, kJacThreads, 0, st>>>(dt, d_col, d_perm, Y, V1, sig, S, VT, U);
    count_launch(2);
    s = cuda_ok(c, cudaGetLastError(), "singular vectors");
  }
  // ---- 5. U = Q (V1; 0)
  if (!s && nv > 0) {
    const bool ok = on_lanes(
        [&](SvdLane& l, int k) {
          const JacJob& t = tab[k];
          return cusolverDnDormqr(l.h, CUBLAS_SIDE_LEFT, CUBLAS_OP_N, t.m, t.n, t.n, T + t.offA,
                                  t.m, tau + t.offTau, U + t.offU, t.m, (double*)l.dwork,
                                  (int)(l.dbytes / sizeof(double)),
                                  qinfo + k) == CUSOLVER_STATUS_SUCCESS;
        },
        [&](int k) { return tab[k].offV >= 0; });
    if (!ok) s = fail(c, DMRG3S_ERR_CUDA, "left singular vectors (ormqr)");
  }
  for (int k = 0; k < nj; ++k) {
    info[k] = conv[k] ? 0 : 1;
    if (!conv[k] && diag && diag->empty())
      *diag = "matrix " + std::to_string(k) + " (" + std::to_string(tab[k].m) + " x " +
              std::to_string(tab[k].n) + ") still had " + std::to_string(hrot[k]) +
              " rotations in sweep " + std::to_string(max_sweeps);
  }
  cudaFreeAsync(dd, st);
  cudaFreeAsync(di, st);
  cudaFreeAsync(dt, st);
  if (ev_in) cudaEventDestroy(ev_in);
  return s;
}

}  // namespace dmrg3s

extern "C" dmrg3s_status dmrg3s_svd(dmrg3s_ctx ctx, int32_t nmat, const int64_t* m,
                                    const int64_t* n, double* A, double* S, double* VT, double* U,
                                    dmrg3s_stream stream) {
  using namespace dmrg3s;
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c) return DMRG3S_ERR_ARG;
  if (nmat < 0 || (nmat > 0 && (!m || !n || !A || !S || !VT)))
    return fail(c, DMRG3S_ERR_ARG, "dmrg3s_svd: null argument or negative count");
  if (nmat == 0) return DMRG3S_OK;
  dmrg3s_status s = use_device(c);
  if (s) return s;
  std::vector<SvdJob> jobs(nmat);
  int64_t oa = 0, os = 0, ov = 0;
  for (int k = 0; k < nmat; ++k) {
    if (n[k] < 1 || m[k] < n[k]) return fail(c, DMRG3S_ERR_ARG, "dmrg3s_svd: need 1 <= n <= m");
    jobs[k].m = m[k];
    jobs[k].n = n[k];
    jobs[k].offA = oa;
    jobs[k].offU = U ? oa : -1;
    jobs[k].offS = os;
    jobs[k].offVT = ov;
    oa += m[k] * n[k];
    os += n[k];
    ov += n[k] * n[k];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<SvdLane> lanes(1);
  std::vector<int> info(nmat, 0);
  std::string diag;
  if (!(s = lane_create(c, &lanes[0]))) {
    s = svd_jacobi(c, lanes, 1, jobs, A, S, VT, U, info.data(), st, &diag);
    if (!s && cudaStreamSynchronize(st) != cudaSuccess)
      s = fail(c, DMRG3S_ERR_CUDA, "dmrg3s_svd: stream synchronisation");
  }
  lane_destroy(&lanes[0]);
  for (int k = 0; !s && k < nmat; ++k)
    if (info[k]) s = fail(c, DMRG3S_ERR_NOT_CONVERGED, "dmrg3s_svd: " + diag);
  return s;
}
