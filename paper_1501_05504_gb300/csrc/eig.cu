// Local eigensolver of DMRG3S: smallest eigenpair of L_{i-1} R_{i+1} W_i M_i =
// lambda M_i (Eq. es-iter, step 1 of Sec. V of arXiv:1501.05504) by Lanczos
// with full reorthogonalisation (classical Gram-Schmidt applied twice).  The
// matrix-vector product is the grouped H_eff contraction; dots and updates
// are FP64 device reductions; the tridiagonal eigenproblem is solved on the
// device.  The host reads back one small struct per iteration to decide
// whether to stop.
#include <cmath>
#include <cstring>

#include "context.hpp"
#include "dmrg3s.h"
#include "kernels.hpp"
#include "vecops.hpp"

namespace dmrg3s {

dmrg3s_status lanczos_run(Context* c, const DevicePlan& heff, const double* Ldata,
                          const double* Rdata, double* x, int64_t n, int kmax, double tol,
                          size_t cursor, cudaStream_t st, double* theta, int* iters,
                          dmrg3s_precision prec) {
  if (kmax < 1 || kmax > 128) return fail(c, DMRG3S_ERR_ARG, "kmax must be in [1, 128]");
  const size_t vbytes = (size_t)n * sizeof(double);
  void *pV, *pw, *ppart, *ph, *palpha, *pbeta, *py, *pn2, *pout;
  dmrg3s_status s;
  if ((s = carve(c, &cursor, vbytes * (kmax + 1), &pV)) || (s = carve(c, &cursor, vbytes, &pw)) ||
      (s = carve(c, &cursor, sizeof(double) * kRedBlocks * (kmax + 1), &ppart)) ||
      (s = carve(c, &cursor, sizeof(double) * (kmax + 1), &ph)) ||
      (s = carve(c, &cursor, sizeof(double) * (kmax + 1), &palpha)) ||
      (s = carve(c, &cursor, sizeof(double) * (kmax + 1), &pbeta)) ||
      (s = carve(c, &cursor, sizeof(double) * (kmax + 1), &py)) ||
      (s = carve(c, &cursor, sizeof(double) * 2, &pn2)) ||
      (s = carve(c, &cursor, sizeof(TridiagOut), &pout)))
    return s;
  double* V = (double*)pV;
  double* w = (double*)pw;
  double* part = (double*)ppart;
  double* h = (double*)ph;
  double* alpha = (double*)palpha;
  double* beta = (double*)pbeta;
  double* y = (double*)py;
  double* nrm2 = (double*)pn2;
  TridiagOut* out = (TridiagOut*)pout;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + heff.host.ws1;
  // tensor-core products: pack the environments once for the whole run
  SplitHints hints;
  if (prec != DMRG3S_FP64) {
    const Plan& hp = heff.host;
    const TcSlots sl = tc_slots(hp);
    const TcStage& t1 = hp.g12.tc;      // the fused H_eff: coefficient-scaled L blocks
    const TcStage& t3 = hp.g3s.tc;
    float* Lp = reinterpret_cast<float*>(ws1 + sl.a1);
    float* Rp = reinterpret_cast<float*>(ws1 + sl.x3);
    launch_pack(heff.g12_packA, (int)t1.packA.size(), t1.tilesA, Ldata, Lp,
                prec == DMRG3S_TF32X3 ? Lp + t1.nA : nullptr, st);
    launch_pack(heff.g3s_packB, (int)t3.packB.size(), t3.tilesB, Rdata, Rp,
                prec == DMRG3S_TF32X3 ? Rp + t3.nB : nullptr, st);
    hints.g1A = true;
    hints.g3B = true;
  }

  // v_0 = x / |x|
  launch_multidot(x, 0, 1, x, n, part, nrm2, nullptr, st);
  cudaMemcpyAsync(c->pinned, nrm2, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "Lanczos start");
  if (!(c->pinned[0] > 0.0)) return fail(c, DMRG3S_ERR_BREAKDOWN, "zero start vector");
  launch_normalise(x, V, n, nrm2, st);

  // Iteration k: w = H v_k was enqueued before; orthogonalise, then solve the
  // tridiagonal problem on the side stream while the main stream already
  // normalises v_{k+1} and applies H to it.  If iteration k turns out to be
  // the last, that product is discarded (its flops are not counted).
  int k = 0;
  TridiagOut res{};
  dmrg3s_status rs = run_plan(c, heff, Ldata, V, ws1, ws2, 1.0, ws2, Rdata, w, st, prec, &hints);
  if (rs != DMRG3S_OK) return fail(c, rs, "H_eff launch failed");
  for (;; ++k) {
    launch_multidot(V, n, k + 1, w, n, part, h, alpha + k, st);   // alpha_k = <v_k, H v_k>
    launch_multi_axpy(V, n, k + 1, h, w, n, st);
    launch_multidot(V, n, k + 1, w, n, part, h, nullptr, st);     // second Gram-Schmidt pass
    launch_multi_axpy(V, n, k + 1, h, w, n, st);
    launch_multidot(w, 0, 1, w, n, part, nrm2, nullptr, st);
    cudaEventRecord(c->ev_ready, st);
    cudaStreamWaitEvent(c->aux, c->ev_ready, 0);
    launch_tridiag_smallest(alpha, beta, k + 1, nrm2, y, out, c->aux);
    cudaMemcpyAsync(c->pinned, out, sizeof(TridiagOut), cudaMemcpyDeviceToHost, c->aux);
    cudaMemcpyAsync(c->pinned + 8, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->aux);
    cudaEventRecord(c->ev_done, c->aux);
    // speculative: the next basis vector and its product
    const bool spec = k + 1 < kmax;
    size_t rec0 = c->prof.recs.size();
    if (spec) {
      launch_normalise(w, V + (int64_t)(k + 1) * n, n, nrm2, st);
      rs = run_plan(c, heff, Ldata, V + (int64_t)(k + 1) * n, ws1, ws2, 1.0, ws2, Rdata, w, st,
                    prec, &hints);
      if (rs != DMRG3S_OK) return fail(c, rs, "H_eff launch failed");
    }
    if (cudaEventSynchronize(c->ev_done) != cudaSuccess)
      return fail(c, DMRG3S_ERR_CUDA, "Lanczos step");
    std::memcpy(&res, c->pinned, sizeof(res));
    int dev_err = 0;
    std::memcpy(&dev_err, c->pinned + 8, sizeof(int));
    if (dev_err) {
      cudaStreamSynchronize(st);
      cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
      return fail(c, DMRG3S_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
    }
    if (res.nan_seen != 0.0) return fail(c, DMRG3S_ERR_NUMERIC, "NaN in the Lanczos recursion");
    const bool conv = res.resid <= tol * std::fmax(1.0, std::fabs(res.theta));
    if (conv || res.beta_last < 1e-14 || k + 1 == kmax) {
      for (size_t r = rec0; r < c->prof.recs.size(); ++r) {   // the discarded product
        c->prof.recs[r].flops = 0.0;
        c->prof.recs[r].bytes = 0.0;
      }
      break;
    }
  }
  // y was written on the side stream
  cudaStreamWaitEvent(st, c->ev_done, 0);
  // Ritz vector x = V y, normalised
  launch_combine_vectors(V, n, k + 1, y, w, n, st);
  launch_multidot(w, 0, 1, w, n, part, nrm2, nullptr, st);
  launch_normalise(w, x, n, nrm2, st);
  if (cudaGetLastError() != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "Lanczos launch failed");
  *theta = res.theta;
  *iters = k + 1;
  return DMRG3S_OK;
}

}  // namespace dmrg3s

using namespace dmrg3s;

extern "C" dmrg3s_status dmrg3s_eigensolve(dmrg3s_ctx ctx, const dmrg3s_env* L,
                                           const dmrg3s_mpo_site* W, const dmrg3s_env* R,
                                           dmrg3s_site* M, int32_t kmax, double tol,
                                           dmrg3s_precision prec, double* lambda, int32_t* iters,
                                           dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !L || !W || !R || !M || !lambda) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  if (prec != DMRG3S_FP64 && prec != DMRG3S_TF32X3 && prec != DMRG3S_TF32)
    return fail(c, DMRG3S_ERR_ARG, "eigensolver precision");
  std::string err;
  EnvLayout le, re;
  MpoLayout w;
  SiteLayout a;
  dmrg3s_status st;
  if ((st = make_env(L, &le, &err)) || (st = make_env(R, &re, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(M, &a, &err)))
    return fail(c, st, err);
  if ((st = check_site_mpo(a, w, &err)) || (st = check_env(le, a.left, w.wl, w.tl, "L", &err)) ||
      (st = check_env(re, a.right, w.wr, w.tr, "R", &err)))
    return fail(c, st, err);
  if (!L->data || !R->data || !M->data) return fail(c, DMRG3S_ERR_ARG, "NULL device data");
  if (a.size == 0) return fail(c, DMRG3S_ERR_SHAPE, "site tensor has no allowed block");
  if ((st = use_device(c))) return st;
  const DevicePlan* p = nullptr;
  if ((st = heff_plan(c, le, w, re, a, &p))) return st;
  size_t cursor = (size_t)plan_ws_doubles(p->host, prec) * sizeof(double);
  int it = 0;
  double theta = 0.0;
  st = lanczos_run(c, *p, L->data, R->data, M->data, a.size, kmax, tol, cursor,
                   reinterpret_cast<cudaStream_t>(stream), &theta, &it, prec);
  if (st != DMRG3S_OK) return st;
  *lambda = theta;
  if (iters) *iters = it;
  return DMRG3S_OK;
}
