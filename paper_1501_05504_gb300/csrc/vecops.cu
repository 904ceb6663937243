// Dense vector kernels of the local eigensolver and the truncation step.
//
// Reductions are deterministic: a fixed grid of kRedBlocks CTAs writes one
// partial sum per CTA (warp-shuffle reduction inside the CTA) and a second
// kernel adds the partials in a fixed order.
#include <cmath>

#include "kernels.hpp"
#include "vecops.hpp"

namespace dmrg3s {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;   // valid in thread 0
}

// h[j] = <V_j, w> for j < k: block (c, j) sums chunk c of vector j (one block
// reduction per block); multidot_final adds the chunk partials of vector j
// in chunk order, so the result is deterministic.
__global__ void __launch_bounds__(kThreads) multidot_partial(const double* __restrict__ V,
                                                             int64_t ldv, const double* __restrict__ w,
                                                             int64_t n, int64_t chunk,
                                                             double* __restrict__ partial) {
  __shared__ double sh[32];
  const int j = blockIdx.y;
  const double* v = V + (int64_t)j * ldv;
  const int64_t e0 = (int64_t)blockIdx.x * chunk;
  const int64_t e1 = e0 + chunk < n ? e0 + chunk : n;
  double acc = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) acc = fma(v[e], w[e], acc);
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = s;
}

__global__ void multidot_final(const double* __restrict__ partial, int nchunk, int k,
                               double* __restrict__ h, double* __restrict__ copy_last) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nchunk; b += blockDim.x) acc += partial[(int64_t)j * nchunk + b];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    h[j] = s;
    if (copy_last && j == k - 1) *copy_last = s;
  }
}

// Double-float numbers (an unevaluated sum hi + lo of two floats, about 44
// significant bits) carry the Sturm counts: GB300 issues FP32 at ~60x its
// FP64 rate, and the count only needs the sign of each pivot. Two-sum is
// Knuth's error-free addition; the quotient takes one correction step with
// an FMA residual (Dekker's double-length division).
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ DF df_sub(DF a, DF b) {
  const float s = a.hi - b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (-b.hi - bb);
  e += a.lo - b.lo;
  const float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float rb = 1.0f / b.hi;
  const float q1 = a.hi * rb;
  const float p = q1 * b.hi;
  const float pe = fmaf(q1, b.hi, -p);
  const float r = (((a.hi - p) - pe) + a.lo) - q1 * b.lo;
  const float q2 = r * rb;
  const float h = q1 + q2;
  return {h, q2 - (h - q1)};
}

// Number of eigenvalues of T smaller than x (Sturm sequence of the LDL^T
// pivots). The matrix arrives shifted and scaled, sa[i] = (alpha_i - c)/s and
// sbb[i] = (beta_{i-1}/s)^2, so every quantity is O(1) and x is (x - c)/s.
__device__ int sturm_count_df(const DF* sa, const DF* sbb, int k, DF x) {
  int cnt = 0;
  DF d = {1.f, 0.f};
  for (int i = 0; i < k; ++i) {
    DF t = df_sub(sa[i], x);
    if (i > 0) t = df_sub(t, df_div(sbb[i], d));
    if (t.hi == 0.f) t = {-1e-30f, 0.f};   // x hit an eigenvalue of a leading block: perturb
    if (t.hi < 0.f) ++cnt;
    d = t;
  }
  return cnt;
}

__device__ void tridiag_vector(const double* alpha, const double* beta, int k, double bl,
                               double theta, double span, double lo, double hi, double* y,
                               TridiagOut* out);

// Multisection: all threads of the block evaluate Sturm counts at equally
// spaced points of the bracket, shrinking it by blockDim.x + 1 per round
// until it reaches the resolution of double-float counts (~1e-13 of the
// Gershgorin span); thread 0 then runs the inverse iteration in FP64 and
// returns the Rayleigh quotient of the vector, which is accurate to FP64
// rounding whatever the width of the bracket was.
// bl = the norm of the new residual vector (stored as beta[k - 1]).
__device__ void tridiag_block(const double* __restrict__ alpha, double* __restrict__ beta, int k,
                              double bl, double* __restrict__ y, TridiagOut* __restrict__ out) {
  __shared__ double sh_lo, sh_hi, sh_span, sh_c;
  __shared__ int sh_bad, sh_first;
  __shared__ DF sa[128], sbb[128];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    double lo = 1e300, hi = -1e300;
    int bad = 0;
    for (int i = 0; i < k; ++i) {
      const double bi = i < k - 1 ? beta[i] : 0.0;
      const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + fabs(bi);
      lo = fmin(lo, alpha[i] - r);
      hi = fmax(hi, alpha[i] + r);
      if (!(alpha[i] == alpha[i])) bad = 1;
    }
    if (!(bl == bl)) bad = 1;
    const double span = fmax(hi - lo, 1e-300);
    sh_lo = lo - 1e-12 * span;
    sh_hi = hi + 1e-12 * span;
    sh_span = span;
    sh_c = 0.5 * (lo + hi);
    sh_bad = bad;
    beta[k - 1] = bl;
  }
  __syncthreads();
  if (sh_bad) {
    if (tid == 0) {
      out->theta = 0.0;
      out->resid = 0.0;
      out->beta_last = bl;
      out->nan_seen = 1.0;
    }
    return;
  }
  const double c = sh_c, inv_s = 1.0 / sh_span;
  for (int i = tid; i < k; i += nt) {
    sa[i] = df_from((alpha[i] - c) * inv_s);
    const double bs = i > 0 ? beta[i - 1] * inv_s : 0.0;
    sbb[i] = df_from(bs * bs);
  }
  __syncthreads();
  for (int round = 0; round < 8; ++round) {
    const double lo = sh_lo, hi = sh_hi;
    const double h = (hi - lo) / (nt + 1);
    if (!(h > 1e-14 * sh_span)) break;
    if (tid == 0) sh_first = nt;
    __syncthreads();
    const DF x = df_from((lo + h * (tid + 1) - c) * inv_s);
    if (sturm_count_df(sa, sbb, k, x) >= 1) atomicMin(&sh_first, tid);
    __syncthreads();
    if (tid == 0) {
      const int f = sh_first;            // first point above the smallest eigenvalue
      sh_hi = f < nt ? lo + h * (f + 1) : hi;
      sh_lo = f > 0 ? lo + h * f : lo;
    }
    __syncthreads();
  }
  if (tid == 0)
    tridiag_vector(alpha, beta, k, bl, 0.5 * (sh_lo + sh_hi), sh_span, sh_lo, sh_hi, y, out);
}

__device__ void tridiag_vector(const double* alpha, const double* beta, int k, double bl,
                               double theta, double span, double lo, double hi, double* y,
                               TridiagOut* out) {
  const int kk = k <= 128 ? k : 128;
  if (kk == 1) {                 // the Ritz vector of a 1x1 matrix
    y[0] = 1.0;
    out->theta = theta;
    out->resid = fabs(bl);
    out->beta_last = bl;
    out->nan_seen = 0.0;
    return;
  }
  // inverse iteration: solve (T - theta I) z = y with a pivoted tridiagonal LU
  // (partial pivoting keeps the elimination stable at the near-singular shift);
  // an exactly zero pivot is replaced by 1e-15 of the matrix scale, which keeps
  // the solution finite (of order 1e15 times the scale) before normalisation.
  // The shift is the same in every sweep, so the matrix is factored once and
  // the pivots are inverted once; a sweep is then two substitutions without
  // divisions (FP64 division is the long pole of this one-thread chain).
  const double tiny = 1e-15 * fmax(span, fmax(fabs(lo), fabs(hi)));
  double dl[128], dd[128], du[128], du2[128];
  int piv[128];
  for (int i = 0; i < kk; ++i) {
    dd[i] = alpha[i] - theta;
    du[i] = i < kk - 1 ? beta[i] : 0.0;
    dl[i] = i < kk - 1 ? beta[i] : 0.0;
    du2[i] = 0.0;
  }
  for (int i = 0; i < kk - 1; ++i) {
    if (fabs(dd[i]) >= fabs(dl[i])) {
      piv[i] = i;
      if (dd[i] == 0.0) dd[i] = tiny;
      const double f = dl[i] / dd[i];
      dl[i] = f;
      dd[i + 1] -= f * du[i];
    } else {
      piv[i] = i + 1;
      const double f = dd[i] / dl[i];
      dd[i] = dl[i];
      dl[i] = f;
      const double t = du[i];
      du[i] = dd[i + 1];
      dd[i + 1] = t - f * dd[i + 1];
      if (i < kk - 2) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
    }
  }
  for (int i = 0; i < kk; ++i) {
    if (dd[i] == 0.0) dd[i] = tiny;
    dd[i] = 1.0 / dd[i];               // dd now holds the inverted pivots
  }
  for (int i = 0; i < kk; ++i) y[i] = 1.0 / sqrt((double)kk);
  for (int sweep = 0; sweep < 3; ++sweep) {
    // forward: apply row interchanges and L
    for (int i = 0; i < kk - 1; ++i) {
      if (piv[i] == i) {
        y[i + 1] -= dl[i] * y[i];
      } else {
        const double t = y[i];
        y[i] = y[i + 1];
        y[i + 1] = t - dl[i] * y[i];
      }
    }
    // back substitution with U (inverted diagonal dd, super du, second super du2)
    y[kk - 1] *= dd[kk - 1];
    if (kk > 1) y[kk - 2] = (y[kk - 2] - du[kk - 2] * y[kk - 1]) * dd[kk - 2];
    for (int i = kk - 3; i >= 0; --i)
      y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) * dd[i];
    // normalise: scale by the largest component first (no overflow in the squares)
    double big = 0.0;
    for (int i = 0; i < kk; ++i) big = fmax(big, fabs(y[i]));
    if (!(big > 0.0) || !(big < 1e308)) {   // degenerate solve: restart from e_0
      for (int i = 0; i < kk; ++i) y[i] = i == 0 ? 1.0 : 0.0;
      continue;
    }
    const double ib = 1.0 / big;
    double nrm = 0.0;
    for (int i = 0; i < kk; ++i) {
      y[i] *= ib;
      nrm += y[i] * y[i];
    }
    const double in = 1.0 / sqrt(nrm);
    for (int i = 0; i < kk; ++i) y[i] *= in;
  }
  // fix the sign: largest component positive (only the subspace is defined)
  int imax = 0;
  for (int i = 1; i < kk; ++i)
    if (fabs(y[i]) > fabs(y[imax])) imax = i;
  if (y[imax] < 0.0)
    for (int i = 0; i < kk; ++i) y[i] = -y[i];
  // Rayleigh quotient y^T T y (y has unit norm): second-order accurate in the
  // error of the vector, so the bracket's width does not limit the Ritz value
  double rq = 0.0;
  for (int i = 0; i < kk; ++i) {
    double ty = alpha[i] * y[i];
    if (i > 0) ty += beta[i - 1] * y[i - 1];
    if (i < kk - 1) ty += beta[i] * y[i + 1];
    rq += y[i] * ty;
  }
  if (rq == rq) theta = rq;
  out->theta = theta;
  out->resid = fabs(bl * y[kk - 1]);
  out->beta_last = bl;
  out->nan_seen = 0.0;
}

__global__ void copy_blocks_kernel(const CopyTask* __restrict__ tasks,
                                   const double* __restrict__ src, double* __restrict__ dst,
                                   const double* __restrict__ scale) {
  const CopyTask t = tasks[blockIdx.x];
  const int n = t.rows * t.cols;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    int r, c;
    if (t.trans) {      // walk the source contiguously
      c = idx / t.rows;
      r = idx % t.rows;
    } else {
      r = idx / t.cols;
      c = idx % t.cols;
    }
    double v = t.trans ? src[t.off_s + (int64_t)c * t.ld_s + r] : src[t.off_s + (int64_t)r * t.ld_s + c];
    if (t.rs >= 0) v *= scale[t.rs + r];
    if (t.cs >= 0) v *= scale[t.cs + c];
    dst[t.off_d + (int64_t)r * t.ld_d + c] = v;
  }
}

// ---- batched Lanczos kernels (see vecops.hpp) ----
constexpr int kLzThreads = 256;
constexpr int kLzWarps = kLzThreads / 32;

// Sum of partial[b * kp + j] over the chunks b of [c0, c0 + nc) in a fixed
// order (lane-strided sums, then the xor tree); every lane returns the sum.
__device__ __forceinline__ double chain_sum(const double* __restrict__ partial, int kp, int c0,
                                            int nc, int j, int lane) {
  double a0 = 0.0, a1 = 0.0;
  int b = lane;
  for (; b + 32 < nc; b += 64) {     // two loads in flight per lane
    const double x0 = partial[(int64_t)(c0 + b) * kp + j];
    const double x1 = partial[(int64_t)(c0 + b + 32) * kp + j];
    a0 += x0;
    a1 += x1;
  }
  if (b < nc) a0 += partial[(int64_t)(c0 + b) * kp + j];
  return warp_sum(a0 + a1);
}

// <v, x> over len elements by one warp (lane-strided), four loads in flight
// per lane; the lanes' partial sums in a fixed order, then the xor tree.
__device__ __forceinline__ double warp_dot(const double* __restrict__ v, const double* x, int len,
                                           int lane) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = lane;
  for (; i + 96 < len; i += 128) {
    const double v0 = v[i], v1 = v[i + 32], v2 = v[i + 64], v3 = v[i + 96];
    a0 = fma(v0, x[i], a0);
    a1 = fma(v1, x[i + 32], a1);
    a2 = fma(v2, x[i + 64], a2);
    a3 = fma(v3, x[i + 96], a3);
  }
  for (; i < len; i += 32) a0 = fma(v[i], x[i], a0);
  return warp_sum((a0 + a1) + (a2 + a3));
}

// x - sum_{j < k1} h[j] V_j[e], the loads of four basis vectors in flight at a
// time (the basis is L2-resident; the loop is latency-bound otherwise).
__device__ __forceinline__ double lz_project(const double* __restrict__ V, int64_t ldv, int k1,
                                             const double* h, int64_t e, double x) {
  int j = 0;
  for (; j + 4 <= k1; j += 4) {
    const double v0 = V[(int64_t)j * ldv + e], v1 = V[(int64_t)(j + 1) * ldv + e];
    const double v2 = V[(int64_t)(j + 2) * ldv + e], v3 = V[(int64_t)(j + 3) * ldv + e];
    x = fma(-h[j], v0, x);
    x = fma(-h[j + 1], v1, x);
    x = fma(-h[j + 2], v2, x);
    x = fma(-h[j + 3], v3, x);
  }
  for (; j < k1; ++j) x = fma(-h[j], V[(int64_t)j * ldv + e], x);
  return x;
}

// The chunk of w is staged in shared memory once; warp q then forms the dot
// products with V_j for j = q, q + 8, ...
__global__ void __launch_bounds__(kLzThreads) lz_dots_kernel(const double* __restrict__ V,
                                                             int64_t ldv, int k1,
                                                             const int* __restrict__ kdev,
                                                             const double* __restrict__ w,
                                                             const LzChunk* __restrict__ chunks,
                                                             double* __restrict__ partial, int kp) {
  extern __shared__ double wsh[];
  if (kdev) k1 = *kdev + 1;
  const LzChunk ch = chunks[blockIdx.x];
  const int len = (int)(ch.e1 - ch.e0);
  for (int i = threadIdx.x; i < len; i += kLzThreads) wsh[i] = w[ch.e0 + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  for (int j = q; j < k1; j += kLzWarps) {
    const double acc = warp_dot(V + (int64_t)j * ldv + ch.e0, wsh, len, lane);
    if (lane == 0) partial[(int64_t)blockIdx.x * kp + j] = acc;
  }
}

__global__ void __launch_bounds__(kLzThreads) lz_update_kernel(
    const double* __restrict__ V, int64_t ldv, int k1, const int* __restrict__ kdev,
    double* __restrict__ w, const LzChunk* __restrict__ chunks, const LzChain* __restrict__ chains,
    const double* __restrict__ partial, int kp, double* __restrict__ alpha,
    double* __restrict__ nrm_partial, int64_t nrm_stride) {
  __shared__ double h[kLzMaxK];
  __shared__ double red[32];
  if (kdev) {
    k1 = *kdev + 1;
    if (nrm_partial) nrm_partial += (int64_t)(*kdev % kLzLag) * nrm_stride;
  }
  const LzChunk ch = chunks[blockIdx.x];
  const LzChain cn = chains[ch.chain];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  for (int j = q; j < k1; j += kLzWarps) {
    const double s = chain_sum(partial, kp, cn.c0, cn.nc, j, lane);
    if (lane == 0) {
      h[j] = s;
      if (alpha && j == k1 - 1 && (int)blockIdx.x == cn.c0) alpha[(int64_t)ch.chain * kp + j] = s;
    }
  }
  __syncthreads();
  double nacc = 0.0;
  for (int64_t e = ch.e0 + threadIdx.x; e < ch.e1; e += kLzThreads) {
    double acc = lz_project(V, ldv, k1, h, e, w[e]);
    if (k1 > 0) w[e] = acc;
    nacc = fma(acc, acc, nacc);
  }
  if (nrm_partial) {
    const double t = block_sum(nacc, red);
    if (threadIdx.x == 0) nrm_partial[blockIdx.x] = t;
  }
}

// The first Gram-Schmidt pass's update fused with the second pass's dots:
// the updated chunk of w stays in shared memory for the dots against V_j.
__global__ void __launch_bounds__(kLzThreads) lz_update_dots_kernel(
    const double* __restrict__ V, int64_t ldv, int k1, double* __restrict__ w,
    const LzChunk* __restrict__ chunks, const LzChain* __restrict__ chains,
    const double* __restrict__ partial, int kp, double* __restrict__ alpha,
    double* __restrict__ partial2, const int* __restrict__ kdev) {
  extern __shared__ double wsh[];
  __shared__ double h[kLzMaxK];
  if (kdev) k1 = *kdev + 1;
  const LzChunk ch = chunks[blockIdx.x];
  const LzChain cn = chains[ch.chain];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  for (int j = q; j < k1; j += kLzWarps) {
    const double s = chain_sum(partial, kp, cn.c0, cn.nc, j, lane);
    if (lane == 0) {
      h[j] = s;
      if (alpha && j == k1 - 1 && (int)blockIdx.x == cn.c0) alpha[(int64_t)ch.chain * kp + j] = s;
    }
  }
  __syncthreads();
  const int len = (int)(ch.e1 - ch.e0);
  for (int i = threadIdx.x; i < len; i += kLzThreads) {
    const int64_t e = ch.e0 + i;
    const double acc = lz_project(V, ldv, k1, h, e, w[e]);
    w[e] = acc;
    wsh[i] = acc;
  }
  __syncthreads();
  for (int j = q; j < k1; j += kLzWarps) {
    const double acc = warp_dot(V + (int64_t)j * ldv + ch.e0, wsh, len, lane);
    if (lane == 0) partial2[(int64_t)blockIdx.x * kp + j] = acc;
  }
}

__global__ void __launch_bounds__(kLzThreads) lz_normalise_kernel(
    const double* __restrict__ x, double* __restrict__ y, const LzChunk* __restrict__ chunks,
    const LzChain* __restrict__ chains, const double* __restrict__ nrm_partial) {
  __shared__ double scale;
  const LzChunk ch = chunks[blockIdx.x];
  if (threadIdx.x < 32) {
    const LzChain cn = chains[ch.chain];
    const double n2 = chain_sum(nrm_partial, 1, cn.c0, cn.nc, 0, threadIdx.x);
    if (threadIdx.x == 0) scale = (n2 > 0.0 && n2 < 1e308) ? 1.0 / sqrt(n2) : 0.0;
  }
  __syncthreads();
  const double sc = scale;
  for (int64_t e = ch.e0 + threadIdx.x; e < ch.e1; e += kLzThreads) y[e] = x[e] * sc;
}

// v_{k+1} = w / |w| (norm partials of iteration k, k from the device
// counter), written into the basis and into the fixed product input vcur.
__global__ void __launch_bounds__(kLzThreads) lz_next_kernel(
    const double* __restrict__ w, double* __restrict__ V, int64_t ldv, const int* __restrict__ kdev,
    double* __restrict__ vcur, const LzChunk* __restrict__ chunks,
    const LzChain* __restrict__ chains, const double* __restrict__ nrm_partial,
    int64_t nrm_stride) {
  __shared__ double scale;
  const int k = *kdev;
  const LzChunk ch = chunks[blockIdx.x];
  if (threadIdx.x < 32) {
    const LzChain cn = chains[ch.chain];
    const double n2 = chain_sum(nrm_partial + (int64_t)(k % kLzLag) * nrm_stride, 1, cn.c0, cn.nc,
                                0, threadIdx.x);
    if (threadIdx.x == 0) scale = (n2 > 0.0 && n2 < 1e308) ? 1.0 / sqrt(n2) : 0.0;
  }
  __syncthreads();
  const double sc = scale;
  double* vn = V + (int64_t)(k + 1) * ldv;
  for (int64_t e = ch.e0 + threadIdx.x; e < ch.e1; e += kLzThreads) {
    const double v = w[e] * sc;
    vn[e] = v;
    vcur[e] = v;
  }
}

__global__ void lz_advance_kernel(int* kdev) { *kdev += 1; }

__global__ void lz_tridiag_kernel(const LzChain* __restrict__ chains, const double* __restrict__ alpha,
                                  double* __restrict__ beta, int kp, int k,
                                  const double* __restrict__ nrm_partial, double* __restrict__ y,
                                  TridiagOut* __restrict__ out) {
  __shared__ double bl;
  const int c = blockIdx.x;
  const LzChain cn = chains[c];
  if (threadIdx.x < 32) {
    const double n2 = chain_sum(nrm_partial, 1, cn.c0, cn.nc, 0, threadIdx.x);
    if (threadIdx.x == 0) bl = sqrt(fmax(n2, 0.0));
  }
  __syncthreads();
  tridiag_block(alpha + (int64_t)c * kp, beta + (int64_t)c * kp, k + 1, bl,
                y + ((int64_t)c * kp + k) * kp, out + (int64_t)k * gridDim.x + c);
}

__global__ void __launch_bounds__(kLzThreads) lz_ritz_kernel(
    const double* __restrict__ V, int64_t ldv, const LzChunk* __restrict__ chunks,
    const LzChain* __restrict__ chains, const int32_t* __restrict__ kstop,
    const double* __restrict__ y, int kp, double* __restrict__ x, double* __restrict__ nrm_partial) {
  __shared__ double red[32];
  const LzChunk ch = chunks[blockIdx.x];
  const int ks = kstop[ch.chain];
  const double* yc = y + ((int64_t)ch.chain * kp + ks) * kp;
  double nacc = 0.0;
  for (int64_t e = ch.e0 + threadIdx.x; e < ch.e1; e += kLzThreads) {
    const double acc = -lz_project(V, ldv, ks + 1, yc, e, 0.0);
    x[e] = acc;
    nacc = fma(acc, acc, nacc);
  }
  const double t = block_sum(nacc, red);
  if (threadIdx.x == 0) nrm_partial[blockIdx.x] = t;
}

}  // namespace

void launch_multidot(const double* V, int64_t ldv, int k, const double* w, int64_t n,
                     double* partial, double* h, double* copy_last, cudaStream_t st) {
  if (k <= 0) return;
  count_launch(2);
  // chunks of at least 2048 elements, at most kRedBlocks of them per vector
  int64_t chunk = (n + kRedBlocks - 1) / kRedBlocks;
  if (chunk < 2048) chunk = 2048;
  chunk = (chunk + kThreads - 1) / kThreads * kThreads;
  int nchunk = (int)((n + chunk - 1) / chunk);
  if (nchunk < 1) nchunk = 1;
  multidot_partial<<<dim3(nchunk, k), kThreads, 0, st>>>(V, ldv, w, n, chunk, partial);
  multidot_final<<<k, 128, 0, st>>>(partial, nchunk, k, h, copy_last);
}

void launch_lz_dots(const double* V, int64_t ldv, int k1, const double* w, const LzChunk* chunks,
                    int nchunks, double* partial, int kp, cudaStream_t st, const int* kdev) {
  if ((!kdev && k1 <= 0) || nchunks <= 0) return;
  count_launch();
  lz_dots_kernel<<<nchunks, kLzThreads, kLzChunkMax * sizeof(double), st>>>(V, ldv, k1, kdev, w,
                                                                             chunks, partial, kp);
}

void launch_lz_update(const double* V, int64_t ldv, int k1, double* w, const LzChunk* chunks,
                      int nchunks, const LzChain* chains, const double* partial, int kp,
                      double* alpha, double* nrm_partial, cudaStream_t st, const int* kdev,
                      int64_t nrm_stride) {
  if (nchunks <= 0) return;
  count_launch();
  lz_update_kernel<<<nchunks, kLzThreads, 0, st>>>(V, ldv, k1, kdev, w, chunks, chains, partial,
                                                   kp, alpha, nrm_partial, nrm_stride);
}

void launch_lz_next(const double* w, double* V, int64_t ldv, const int* kdev, double* vcur,
                    const LzChunk* chunks, int nchunks, const LzChain* chains,
                    const double* nrm_partial, int64_t nrm_stride, cudaStream_t st) {
  if (nchunks <= 0) return;
  count_launch();
  lz_next_kernel<<<nchunks, kLzThreads, 0, st>>>(w, V, ldv, kdev, vcur, chunks, chains,
                                                 nrm_partial, nrm_stride);
}

void launch_lz_advance(int* kdev, cudaStream_t st) {
  count_launch();
  lz_advance_kernel<<<1, 1, 0, st>>>(kdev);
}

void launch_lz_update_dots(const double* V, int64_t ldv, int k1, double* w, const LzChunk* chunks,
                           int nchunks, const LzChain* chains, const double* partial, int kp,
                           double* alpha, double* partial2, cudaStream_t st, const int* kdev) {
  if (nchunks <= 0 || (!kdev && k1 <= 0)) return;
  count_launch();
  lz_update_dots_kernel<<<nchunks, kLzThreads, kLzChunkMax * sizeof(double), st>>>(
      V, ldv, k1, w, chunks, chains, partial, kp, alpha, partial2, kdev);
}

void launch_lz_normalise(const double* x, double* y, const LzChunk* chunks, int nchunks,
                         const LzChain* chains, const double* nrm_partial, cudaStream_t st) {
  if (nchunks <= 0) return;
  count_launch();
  lz_normalise_kernel<<<nchunks, kLzThreads, 0, st>>>(x, y, chunks, chains, nrm_partial);
}

void launch_lz_tridiag(const LzChain* chains, int nchains, const double* alpha, double* beta,
                       int kp, int k, const double* nrm_partial, double* y, TridiagOut* out,
                       cudaStream_t st) {
  if (nchains <= 0) return;
  count_launch();
  lz_tridiag_kernel<<<nchains, 256, 0, st>>>(chains, alpha, beta, kp, k, nrm_partial, y, out);
}

void launch_lz_ritz(const double* V, int64_t ldv, const LzChunk* chunks, int nchunks,
                    const LzChain* chains, const int32_t* kstop, const double* y, int kp,
                    double* x, double* nrm_partial, cudaStream_t st) {
  if (nchunks <= 0) return;
  count_launch();
  lz_ritz_kernel<<<nchunks, kLzThreads, 0, st>>>(V, ldv, chunks, chains, kstop, y, kp, x,
                                                 nrm_partial);
}

void launch_copy_blocks(const CopyTask* tasks, int ntasks, const double* src, double* dst,
                        const double* scale, cudaStream_t st) {
  if (ntasks <= 0) return;
  count_launch();
  copy_blocks_kernel<<<ntasks, 256, 0, st>>>(tasks, src, dst, scale);
}

}  // namespace dmrg3s
