// Dense vector kernels of the local eigensolver (Lanczos, step 1 of Sec. V of
// arXiv:1501.05504) and of the truncation step.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>
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

// Result of the smallest eigenpair of a symmetric tridiagonal Lanczos matrix
// of order k (diagonal alpha, off-diagonal beta[0..k-2]), solved in one CTA:
// Sturm multisection (double-float counts) brackets the eigenvalue, one
// thread runs inverse iteration for the eigenvector and returns its Rayleigh
// quotient; beta[k-1] is set to the norm of the new residual vector.
struct TridiagOut {
  double theta, resid, beta_last, nan_seen;
};

// ---- Lanczos over a batch of independent problems ("chains") ----
// The vectors of all chains are stored back to back: chain c owns elements
// [off, off + n) of every vector (off a multiple of 32).  The vector space is
// cut into chunks (one CTA each) that never straddle two chains; every
// reduction writes one partial per chunk and is finished by summing the
// chain's partials in chunk order (lane-strided, then a fixed shuffle tree),
// so every CTA that needs a chain's sum computes the identical value.
struct LzChunk {
  int64_t e0, e1;       // element range [e0, e1)
  int32_t chain, pad;
};
struct LzChain {
  int64_t off, n;       // element range of the chain
  int32_t c0, nc;       // its chunks [c0, c0 + nc)
};
constexpr int kLzMaxK = 129;   // most basis vectors of one run (kmax <= 128, plus one)
constexpr int kLzChunkMax = 4096;   // most elements of one chunk
constexpr int kLzLag = 3;           // rotating norm-partial buffers of the iterations in flight

// Chunks of `ranges` (one (off, n) per chain): each chain's range cut into
// about equal chunks of at most kLzChunkMax elements, `target` chunks in all
// where the sizes allow (a chain of n elements gets at least one chunk).
inline void lz_layout(const std::vector<std::pair<int64_t, int64_t>>& ranges, int target,
                      std::vector<LzChunk>* chunks, std::vector<LzChain>* chains) {
  int64_t total = 0;
  for (auto& r : ranges) total += r.second;
  int64_t len = target > 0 ? (total + target - 1) / target : total;
  len = (len + 31) / 32 * 32;
  if (len < 256) len = 256;
  if (len > kLzChunkMax) len = kLzChunkMax;
  chunks->clear();
  chains->clear();
  for (size_t c = 0; c < ranges.size(); ++c) {
    LzChain cn{};
    cn.off = ranges[c].first;
    cn.n = ranges[c].second;
    cn.c0 = (int32_t)chunks->size();
    const int64_t nch = cn.n > 0 ? (cn.n + len - 1) / len : 0;
    for (int64_t b = 0; b < nch; ++b) {
      LzChunk ch{};
      ch.e0 = cn.off + cn.n * b / nch;
      ch.e1 = cn.off + cn.n * (b + 1) / nch;
      ch.chain = (int32_t)c;
      chunks->push_back(ch);
    }
    cn.nc = (int32_t)(chunks->size() - cn.c0);
    chains->push_back(cn);
  }
}

// Device-counter form: the kernels below that take `kdev` (non-null) read the
// iteration k from that device word instead of their k1 argument (k1 = k + 1),
// so that one captured launch sequence serves every iteration.
//
// partial[b * kp + j] = <V_j, w> over chunk b, for j < k1 (V_j = V + j * ldv).
void launch_lz_dots(const double* V, int64_t ldv, int k1, const double* w, const LzChunk* chunks,
                    int nchunks, double* partial, int kp, cudaStream_t st,
                    const int* kdev = nullptr);
// One Gram-Schmidt pass: h_j = (chain sum of partial[., j]), w -= sum_{j<k1} h_j V_j.
// alpha (optional): alpha[chain * kp + k1 - 1] = h_{k1-1} (the Lanczos alpha_k).
// nrm_partial (optional): the chunk's sum of squares of the updated w.
// k1 = 0 leaves w unchanged and only forms nrm_partial.  With kdev, the norm
// partials go to nrm_partial + (k % kLzLag) * nrm_stride.
void launch_lz_update(const double* V, int64_t ldv, int k1, double* w, const LzChunk* chunks,
                      int nchunks, const LzChain* chains, const double* partial, int kp,
                      double* alpha, double* nrm_partial, cudaStream_t st,
                      const int* kdev = nullptr, int64_t nrm_stride = 0);
// v_{k+1} = w / |w| into V + (k + 1) ldv and into vcur, k = *kdev, the norm
// partials at nrm_partial + (k % kLzLag) * nrm_stride (zeros for a problem
// whose squared norm is not positive and finite).
void launch_lz_next(const double* w, double* V, int64_t ldv, const int* kdev, double* vcur,
                    const LzChunk* chunks, int nchunks, const LzChain* chains,
                    const double* nrm_partial, int64_t nrm_stride, cudaStream_t st);
// *kdev += 1 (one thread).
void launch_lz_advance(int* kdev, cudaStream_t st);
// The update of one pass followed by the dots of the next: as launch_lz_update
// (without the norm) and then launch_lz_dots of the updated w into partial2
// (which must not be `partial`).
void launch_lz_update_dots(const double* V, int64_t ldv, int k1, double* w, const LzChunk* chunks,
                           int nchunks, const LzChain* chains, const double* partial, int kp,
                           double* alpha, double* partial2, cudaStream_t st,
                           const int* kdev = nullptr);
// y[e] = x[e] / sqrt(chain sum of nrm_partial); a chain whose squared norm is
// not positive and finite gets zeros.
void launch_lz_normalise(const double* x, double* y, const LzChunk* chunks, int nchunks,
                         const LzChain* chains, const double* nrm_partial, cudaStream_t st);
// Smallest eigenpair of every chain's tridiagonal Lanczos matrix of order
// k + 1 (one CTA per chain; the algorithm above):
// beta[c * kp + k] = sqrt(chain sum of nrm_partial), the Ritz vector into
// y + (c * kp + k) * kp, the result into out[k * nchains + c].
void launch_lz_tridiag(const LzChain* chains, int nchains, const double* alpha, double* beta,
                       int kp, int k, const double* nrm_partial, double* y, TridiagOut* out,
                       cudaStream_t st);
// Ritz vectors: x[e] = sum_{j <= kstop[c]} y[(c * kp + kstop[c]) * kp + j] V_j[e] for the
// chain c of element e, and the chunk's sum of squares of x into nrm_partial.
void launch_lz_ritz(const double* V, int64_t ldv, const LzChunk* chunks, int nchunks,
                    const LzChain* chains, const int32_t* kstop, const double* y, int kp,
                    double* x, double* nrm_partial, cudaStream_t st);

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
