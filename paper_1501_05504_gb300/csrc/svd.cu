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
// round is one warp and one launch runs a round of every matrix of the batch;
// one sweep (a launch per round) is a CUDA graph.  A matrix with no rotation
// in a sweep is converged and its warps exit at once in later sweeps.
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
  int32_t m, n, npad, pair0;          // pair0: first pair of the matrix in a round launch
  int32_t col0, pad;                  // first column of the matrix in the batch numbering
  double tol2;                        // the square of the pair tolerance
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

// The rotation (c, s) of a pair with Gram entries alpha = saa, beta = sbb,
// gamma = sab: t = tan(theta) the smaller root of t^2 + 2 zeta t - 1 = 0,
// zeta = (beta - alpha) / (2 gamma), c = 1 / sqrt(1 + t^2), s = c t.  GB300
// issues FP64 at 1/64 of its FP32 rate, and a division or square root in
// FP64 is a long chain of such instructions, so the angle is computed in
// FP32 on (beta - alpha, 2 gamma) scaled by a common power of two (so that
// neither underflows nor overflows), and (c, s) is then made orthonormal to
// FP64 accuracy by two Newton steps on c^2 + s^2 = 1 (FP64 multiply-adds
// only).  The angle carries FP32 rounding (~1e-7 relative): the rotated pair
// is orthogonal to ~1e-7 of its former cosine rather than exactly, which the
// next sweep removes; the rotation itself is orthogonal to FP64 rounding, so
// the singular values are unaffected.
__device__ __forceinline__ void jacobi_rotation(double saa, double sbb, double sab, double* c,
                                                double* s) {
  const double d = sbb - saa, g2 = 2.0 * sab;
  const double big = fmax(fabs(d), fabs(g2));
  // 2^-e with e the binary exponent of big (a normal number here)
  const long long eb = (__double_as_longlong(big) >> 52) & 0x7ff;
  const double scale = __longlong_as_double((long long)(2046 - eb) << 52);
  const double ds = d * scale, gs = g2 * scale;   // the larger magnitude in [1, 2)
  const float df = (float)ds, gf = (float)gs;
  double t;
  if (fabs(ds) > 1048576.0 * fabs(gs)) {
    // |zeta| > 2^20: t = 1 / (2 zeta) = gamma / (beta - alpha) to FP32 rounding, in
    // FP64 (it may be far below the FP32 range) with an FP32 reciprocal of ds
    t = 0.5 * gs * (double)(1.0f / df);
  } else {
    const float z = df / gf;
    t = (double)(copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f))));
  }
  const float tf = (float)t;
  const float c32 = rsqrtf(fmaf(tf, tf, 1.0f));
  double cc = c32, ss = (double)c32 * t;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double r = fma(-0.5, fma(cc, cc, ss * ss), 1.5);
    cc *= r;
    ss *= r;
  }
  *c = cc;
  *s = ss;
}

// Advances the sweep counter read by the round kernels (first node of a sweep).
__global__ void jac_next_sweep_kernel(int* sweep) { *sweep += 1; }

// Sums of three per-lane values over the warp, returned to every lane with
// the same bits in every lane.  The first two levels exchange halves of the
// values a lane carries (the lower 16 lanes go on with x and y, the upper
// with z and a zero; then each group of 8 with one of those), so the five
// levels take 6 FP64 additions instead of the 15 of a butterfly per value;
// the last three levels are a butterfly within each group of 8 lanes, whose
// lanes then hold identical sums (IEEE addition commutes bit for bit).
__device__ __forceinline__ void warp_sum3(double& x, double& y, double& z) {
  const int lane = threadIdx.x & 31;
  const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
  const double w = 0.0;
  const double a = (hi16 ? z : x) + __shfl_xor_sync(0xffffffffu, hi16 ? x : z, 16);
  const double b = (hi16 ? w : y) + __shfl_xor_sync(0xffffffffu, hi16 ? y : w, 16);
  double c = (hi8 ? b : a) + __shfl_xor_sync(0xffffffffu, hi8 ? a : b, 8);
  for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  x = __shfl_sync(0xffffffffu, c, 0);    // lanes 0-7: the sum of x
  y = __shfl_sync(0xffffffffu, c, 8);    // lanes 8-15: of y
  z = __shfl_sync(0xffffffffu, c, 16);   // lanes 16-23: of z
}

// One round r of the current sweep for every matrix: one warp per pair,
// kJacPairsPerCta pairs per CTA.  rot[s * njobs + job] counts the rotations
// of sweep s.  GB300 runs an FP64 warp instruction in ~64 cycles of a
// sub-partition, so the round is priced in FP64 instructions: a warp per
// pair does the pair's three dot products and its rotation with the same
// count as a CTA would, but reduces once instead of once per warp, and every
// lane computes the (identical) rotation itself, with no shared memory, CTA
// barrier or single-thread step.  The first kJacCache elements of each
// lane's share stay in registers between the dot products and the rotation.
constexpr int kJacPairsPerCta = 4;
constexpr int kJacCache = 8;
__global__ void __launch_bounds__(32 * kJacPairsPerCta)
jac_round_kernel(const JacJob* __restrict__ jobs, const int* __restrict__ pair_job, int npairs,
                 int njobs, int r, const int* __restrict__ sweep, int* __restrict__ rot,
                 double* __restrict__ Y, double* __restrict__ V) {
  const int p = blockIdx.x * kJacPairsPerCta + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= npairs) return;
  const int sw = *sweep;
  if (sw < 0 || sw >= kJacobiMaxSweeps) return;
  const int jb = pair_job[p];
  if (sw > 0 && rot[(sw - 1) * njobs + jb] == 0) return;   // converged in the previous sweep
  const JacJob J = jobs[jb];
  const int N = J.npad - 1;
  if (r >= N) return;
  const int k = p - J.pair0;
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
    const int i = lane + e * 32;
    ua[e] = i < n ? ya[i] : 0.0;
    ub[e] = i < n ? yb[i] : 0.0;
    saa = fma(ua[e], ua[e], saa);
    sbb = fma(ub[e], ub[e], sbb);
    sab = fma(ua[e], ub[e], sab);
  }
  for (int i = lane + kJacCache * 32; i < n; i += 32) {
    const double u = ya[i], v = yb[i];
    saa = fma(u, u, saa);
    sbb = fma(v, v, sbb);
    sab = fma(u, v, sab);
  }
  warp_sum3(saa, sbb, sab);
  // zero columns and NaN leave the pair unrotated (NaN reaches the singular values)
  if (!(saa > 0.0 && sbb > 0.0 && sab * sab > J.tol2 * saa * sbb)) return;
  double cs, sn;
  jacobi_rotation(saa, sbb, sab, &cs, &sn);
  if (lane == 0) atomicAdd(rot + sw * njobs + jb, 1);
#pragma unroll
  for (int e = 0; e < kJacCache; ++e) {
    const int i = lane + e * 32;
    if (i < n) {
      ya[i] = cs * ua[e] - sn * ub[e];
      yb[i] = sn * ua[e] + cs * ub[e];
    }
  }
  for (int i = lane + kJacCache * 32; i < n; i += 32) {
    const double u = ya[i], v = yb[i];
    ya[i] = cs * u - sn * v;
    yb[i] = sn * u + cs * v;
  }
  if (J.offV >= 0) {
    double* va = V + J.offV + (int64_t)a * n;
    double* vb = V + J.offV + (int64_t)b * n;
    for (int i = lane; i < n; i += 32) {
      const double u = va[i], v = vb[i];
      va[i] = cs * u - sn * v;
      vb[i] = sn * u + cs * v;
    }
  }
}

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
  std::vector<int> pair_job, col_job;
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
    t.pair0 = (int32_t)pair_job.size();
    t.col0 = (int32_t)col_job.size();
    t.pad = 0;
    const double tol = std::max(std::sqrt((double)t.n), 32.0) * DBL_EPSILON;
    t.tol2 = tol * tol;
    pair_job.insert(pair_job.end(), t.npad / 2, k);
    col_job.insert(col_job.end(), t.n, k);
    maxr = std::max(maxr, t.npad - 1);
  }
  const int npair = (int)pair_job.size(), ncol = (int)col_job.size();
  const int ncta = (npair + kJacPairsPerCta - 1) / kJacPairsPerCta;
  int64_t na = 0;   // extent of the A buffer used by the jobs
  for (const JacJob& t : tab) na = std::max(na, t.offA + (int64_t)t.m * t.n);
  // ---- device buffers: doubles [tau | Y | V1 | sigma | column norms | T = A P],
  //      ints [pair_job | col_job | perm | rot | sweep | qinfo]
  const int64_t nd = ntau + ny + nv + 2 * (int64_t)ncol + na;
  const int64_t ni = npair + 2 * (int64_t)ncol + (int64_t)kJacobiMaxSweeps * nj + 1 + nj;
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
  int* d_pair = di;
  int* d_col = d_pair + npair;
  int* d_perm = d_col + ncol;
  int* rot = d_perm + ncol;
  int* d_sweep = rot + (int64_t)kJacobiMaxSweeps * nj;
  int* qinfo = d_sweep + 1;
  cudaMemcpyAsync(dt, tab.data(), tab.size() * sizeof(JacJob), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_pair, pair_job.data(), pair_job.size() * sizeof(int), cudaMemcpyHostToDevice, st);
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
  // ---- 3. sweeps: one CUDA graph of (sweep counter, rounds 0 .. maxr-1)
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  if (!s && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
      cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    jac_next_sweep_kernel<<<1, 1, 0, cap>>>(d_sweep);
    for (int r = 0; r < maxr; ++r)
      jac_round_kernel<<<ncta, 32 * kJacPairsPerCta, 0, cap>>>(dt, d_pair, npair, nj, r, d_sweep,
                                                              rot, Y, V1);
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
      jac_next_sweep_kernel<<<1, 1, 0, st>>>(d_sweep);
      for (int r = 0; r < maxr; ++r)
        jac_round_kernel<<<ncta, 32 * kJacPairsPerCta, 0, st>>>(dt, d_pair, npair, nj, r, d_sweep,
                                                              rot, Y, V1);
      s = cuda_ok(c, cudaGetLastError(), "Jacobi sweep");
    }
    count_launch(maxr + 1);
    if (id >= 0) pr.end(id, st);
    if (s) break;
    if ((s = cuda_ok(c, cudaMemcpyAsync(hrot.data(), rot + (int64_t)sw * nj, nj * sizeof(int),
                                        cudaMemcpyDeviceToHost, st), "Jacobi rotations")) ||
        (s = cuda_ok(c, cudaStreamSynchronize(st), "Jacobi sweep")))
      break;
    // algorithmic cost of the sweep: a pair test reads two columns (16n bytes)
    // for three dot products (6n flops); a rotation of a column pair of Y and
    // of V1 takes 6n flops each and writes 16n bytes each (V1 also read)
    double fl = 0.0, by = 0.0;
    bool more = false;
    for (int k = 0; k < nj; ++k) {
      if (!active[k]) continue;
      const double n = tab[k].n, pairs = 0.5 * n * (n - 1.0);
      const bool v = tab[k].offV >= 0;
      fl += pairs * 6.0 * n + hrot[k] * 6.0 * n * (v ? 2.0 : 1.0);
      by += pairs * 16.0 * n + hrot[k] * 16.0 * n * (v ? 3.0 : 1.0);
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
      pr.recs[id].launches = maxr + 1;
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
