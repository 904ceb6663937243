// Dense vector kernels of the local eigensolver (Lanczos, step 1 of Sec. V of
// arXiv:1501.05504) and of the truncation step.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dmrg3s {

// Most chunks a vector is split into by the reductions (two per SM of the
// 152-SM GB300).
constexpr int kRedBlocks = 304;

// h[j] = <V_j, w> for j < k with V_j = V + j * ldv.  Deterministic two-pass
// reduction: one CTA per (chunk of >= 2048 elements, vector) writes a partial
// sum into `partial` (room for kRedBlocks * k doubles), then one CTA per
// vector adds its partials in chunk order.  When `copy_last` is non-null,
// h[k-1] is also stored there (the Lanczos alpha_k).
void launch_multidot(const double* V, int64_t ldv, int k, const double* w, int64_t n,
                     double* partial, double* h, double* copy_last, cudaStream_t st);

// w -= sum_{j<k} h[j] V_j
void launch_multi_axpy(const double* V, int64_t ldv, int k, const double* h, double* w, int64_t n,
                       cudaStream_t st);

// y = sum_{j<k} c[j] V_j    (c on the device)
void launch_combine_vectors(const double* V, int64_t ldv, int k, const double* c, double* y,
                            int64_t n, cudaStream_t st);

// y = x / sqrt(*nrm2)   (nrm2 on the device)
void launch_normalise(const double* x, double* y, int64_t n, const double* nrm2, cudaStream_t st);

// Smallest eigenpair of the symmetric tridiagonal Lanczos matrix of order k
// (diagonal alpha, off-diagonal beta[0..k-2]) in one CTA: Sturm multisection
// (double-float counts) brackets the eigenvalue, one thread runs inverse
// iteration for the eigenvector and returns its Rayleigh quotient.
// beta[k-1] is set to sqrt(*nrm2) (the norm of the new residual vector).
struct TridiagOut {
  double theta, resid, beta_last, nan_seen;
};
void launch_tridiag_smallest(const double* alpha, double* beta, int k, const double* nrm2,
                             double* y, TridiagOut* out, cudaStream_t st);

// Copy of rectangular blocks with optional transpose and row/column scaling:
//   dst[off_d + r*ld_d + c] = src(r, c) * rs[r] * cs[c]
// with src(r, c) = src[off_s + r*ld_s + c] or, transposed, src[off_s + c*ld_s + r];
// rs / cs are indexes into `scale` (-1 = no scaling) offset by r / c.
struct CopyTask {
  int64_t off_s, off_d;
  int32_t rows, cols, ld_s, ld_d;
  int32_t trans, rs, cs, pad;
};
void launch_copy_blocks(const CopyTask* tasks, int ntasks, const double* src, double* dst,
                        const double* scale, cudaStream_t st);

}  // namespace dmrg3s
