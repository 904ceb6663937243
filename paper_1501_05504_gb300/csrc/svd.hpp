// FP64 SVD of a batch of column-major matrices: the factorisation of the
// truncation step of the local update (Sec. IV A, Sec. V step 4).
//
// Each matrix A (m x n, m >= n), its columns ordered by descending norm
// (A P), is factorised A P = Q R by cuSOLVER's Householder QR; R^T is then
// orthogonalised by the one-sided (Hestenes) Jacobi method in this library's
// kernels, R^T V1 = W with orthogonal columns, which gives R^T = U1 S V1^T
// (U1 = W S^-1) and
//   A = (Q V1) S (P U1)^T:
// the right singular vectors of A are the normalised columns of W, permuted
// back, the left ones Q V1 (formed only when asked for).
#pragma once

#include <cusolverDn.h>

#include <cstdint>
#include <string>
#include <vector>

#include "context.hpp"

namespace dmrg3s {

// One concurrent cuSOLVER lane: its own handle, stream and workspaces.
struct SvdLane {
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t p = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  void* dwork = nullptr;
  size_t dbytes = 0;
  std::vector<char> hwork;
};
dmrg3s_status lane_create(Context* c, SvdLane* w);
void lane_destroy(SvdLane* w);

// One matrix of a batch.  A (m x n, ld m, m >= n >= 1) at element offset offA
// of the batch's A buffer.  Results: S (n, descending) at offS; VT (n x n,
// ld n, row c = right singular vector c) at offVT; U (m x n, ld m, column c =
// left singular vector c) at offU, or not formed when offU < 0.  Singular
// vectors of a zero singular value: VT row zero, U column an orthonormal
// completion.
struct SvdJob {
  int64_t m = 0, n = 0, offA = 0, offS = 0, offVT = 0, offU = -1;
};

// Jacobi sweeps allowed before a matrix counts as not converged: at most
// kJacobiMaxSweeps, fewer when the environment variable DMRG3S_JACOBI_SWEEPS
// (1 .. kJacobiMaxSweeps) is set.
constexpr int kJacobiMaxSweeps = 40;
int jacobi_max_sweeps();

// Factorises every job; A is only read (the factorisation works on a copy).
// `lanes[0 .. nlanes)` run the QR factorisations (and Q V1) concurrently
// after the work already queued on `st`; `st` waits for all results.
// info[k] (host) = 0, or 1 when job k did not converge within the sweep
// limit (its outputs are then invalid; *diag, when given, names the first
// such job; *sweeps, when given, receives the number of sweeps run).
// Synchronises `st` once per sweep.  Profiling (kind
// kProfJacobi) records each sweep's rounds with the flops of its pair tests
// and rotations.
dmrg3s_status svd_jacobi(Context* c, std::vector<SvdLane>& lanes, int nlanes,
                         const std::vector<SvdJob>& jobs, double* A, double* S, double* VT,
                         double* U, int* info, cudaStream_t st, std::string* diag = nullptr,
                         int* sweeps = nullptr);

}  // namespace dmrg3s
