// Local eigensolver of DMRG3S: smallest eigenpair of L_{i-1} R_{i+1} W_i M_i =
// lambda M_i (Eq. es-iter, step 1 of Sec. V of arXiv:1501.05504) by Lanczos
// with full reorthogonalisation (classical Gram-Schmidt applied twice).  The
// matrix-vector product is the grouped H_eff contraction; dots and updates
// are FP64 device reductions; the tridiagonal eigenproblem is solved on the
// device.  The host reads back one small struct per problem and iteration to
// decide whether to stop, one iteration behind the device.  Several
// independent problems (the chains of a batch) run in one recursion, each
// stage one launch over all of them.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "context.hpp"
#include "dmrg3s.h"
#include "kernels.hpp"
#include "vecops.hpp"

namespace dmrg3s {

dmrg3s_status pinned_reserve(Context* c, size_t n) {
  if (c->pinned_big_n >= n) return DMRG3S_OK;
  if (c->pinned_big) {
    cudaFreeHost(c->pinned_big);
    c->pinned_big = nullptr;
    c->pinned_big_n = 0;
  }
  const size_t want = n < 4096 ? 4096 : n;
  if (cudaMallocHost(&c->pinned_big, want * sizeof(double)) != cudaSuccess)
    return fail(c, DMRG3S_ERR_CUDA, "pinned read-back area");
  c->pinned_big_n = want;
  return DMRG3S_OK;
}

// Iteration k of every problem, on the main stream:
//   two classical Gram-Schmidt passes of w = H v_k against v_0 .. v_k in three
//   launches (dots; update fused with the second pass's dots; update with
//   the partial norms of w); the first pass's last coefficient is alpha_k;
//   v_{k+1} = w / |w|; w = H v_{k+1};
// then, on the side stream, the tridiagonal solve of order k + 1 and the copy
// of its results to the host.  The host reads iteration k's results only
// after it has enqueued iteration k + 2, so the device never waits for the
// host's stopping decision; a problem that has stopped keeps being iterated
// (its results are no longer read) until every problem has stopped, and the
// products of the iterations past the last stop are discarded (their flops
// are not counted).
dmrg3s_status lanczos_batch(Context* c, const DevicePlan& heff, const double* Ldata,
                            const double* Rdata, double* X, int64_t ldx,
                            const std::vector<LzSpec>& probs, size_t cursor, cudaStream_t st,
                            dmrg3s_precision prec, std::vector<double>* theta,
                            std::vector<int>* iters) {
  const int np = (int)probs.size();
  if (np < 1) return fail(c, DMRG3S_ERR_ARG, "no eigenproblem");
  int kmax = 0;
  for (const LzSpec& p : probs) {
    if (p.kmax < 1 || p.kmax > 128) return fail(c, DMRG3S_ERR_ARG, "kmax must be in [1, 128]");
    if (p.off < 0 || p.n < 1 || p.off % 32 != 0 || p.off + p.n > ldx)
      return fail(c, DMRG3S_ERR_ARG, "eigenproblem vector range");
    kmax = std::max(kmax, p.kmax);
  }
  const int kp = kmax + 1;
  const int64_t ldv = (ldx + 31) / 32 * 32;
  std::vector<std::pair<int64_t, int64_t>> ranges(np);
  for (int i = 0; i < np; ++i) ranges[i] = {probs[i].off, probs[i].n};
  std::vector<LzChunk> hch;
  std::vector<LzChain> hcn;
  // about one chunk per SM: few partials per problem to finish the sums
  // from, several elements per thread
  lz_layout(ranges, plan_ctas(), &hch, &hcn);
  const int nchunks = (int)hch.size();
  void *pV, *pw, *pvc, *ppart, *pnp, *palpha, *pbeta, *py, *pout, *pch, *pcn, *pks, *pk;
  dmrg3s_status s;
  if ((s = carve(c, &cursor, sizeof(double) * ldv * kp, &pV)) ||
      (s = carve(c, &cursor, sizeof(double) * ldv, &pw)) ||
      (s = carve(c, &cursor, sizeof(double) * ldv, &pvc)) ||
      (s = carve(c, &cursor, sizeof(double) * nchunks * kp * 2, &ppart)) ||
      (s = carve(c, &cursor, sizeof(double) * nchunks * (kLzLag + 1), &pnp)) ||
      (s = carve(c, &cursor, sizeof(double) * np * kp, &palpha)) ||
      (s = carve(c, &cursor, sizeof(double) * np * kp, &pbeta)) ||
      (s = carve(c, &cursor, sizeof(double) * np * kp * kp, &py)) ||
      (s = carve(c, &cursor, sizeof(TridiagOut) * np * kp, &pout)) ||
      (s = carve(c, &cursor, sizeof(LzChunk) * nchunks, &pch)) ||
      (s = carve(c, &cursor, sizeof(LzChain) * np, &pcn)) ||
      (s = carve(c, &cursor, sizeof(int32_t) * np, &pks)) ||
      (s = carve(c, &cursor, sizeof(int), &pk)))
    return s;
  // read-back slots: kLzLag iterations' results (4 doubles per problem) and the error word
  const size_t slot = (size_t)np * 4 + 2;
  if ((s = pinned_reserve(c, kLzLag * slot + (size_t)nchunks))) return s;
  double* V = (double*)pV;
  double* w = (double*)pw;
  double* vcur = (double*)pvc;     // the vector the product reads: v_k
  double* part = (double*)ppart;
  double* part2 = part + (int64_t)nchunks * kp;
  double* nrm = (double*)pnp;      // kLzLag rotating norm-partial buffers, then one more
  double* nrm_x = nrm + (int64_t)kLzLag * nchunks;
  double* alpha = (double*)palpha;
  double* beta = (double*)pbeta;
  double* y = (double*)py;
  TridiagOut* out = (TridiagOut*)pout;
  LzChunk* dch = (LzChunk*)pch;
  LzChain* dcn = (LzChain*)pcn;
  int32_t* dks = (int32_t*)pks;
  int* kdev = (int*)pk;
  if (cudaMemcpyAsync(dch, hch.data(), sizeof(LzChunk) * nchunks, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(dcn, hcn.data(), sizeof(LzChain) * np, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return fail(c, DMRG3S_ERR_CUDA, "Lanczos tables");
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
  double* pin = c->pinned_big;

  // v_0 = x / |x| for every problem (a zero start vector is an error)
  launch_lz_update(nullptr, ldv, 0, X, dch, nchunks, dcn, nullptr, kp, nullptr, nrm_x, st);
  cudaMemcpyAsync(pin, nrm_x, sizeof(double) * nchunks, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "Lanczos start");
  for (int i = 0; i < np; ++i) {
    double n2 = 0.0;
    for (int b = 0; b < hcn[i].nc; ++b) n2 += pin[hcn[i].c0 + b];
    if (!(n2 > 0.0)) return fail(c, DMRG3S_ERR_BREAKDOWN, "zero start vector");
  }
  launch_lz_normalise(X, V, dch, nchunks, dcn, nrm_x, st);
  cudaMemcpyAsync(vcur, V, sizeof(double) * ldv, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(kdev, 0, sizeof(int), st);

  std::vector<int> kstop(np, -1);
  theta->assign(np, 0.0);
  iters->assign(np, 0);
  int nstopped = 0;
  // an error after the recursion has started waits for both streams (the
  // side stream still writes into the workspace the caller reuses)
  auto bail = [&](dmrg3s_status r) {
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(c->aux);
    return r;
  };
  // profiler records of the product that builds on iteration k (index k + 1)
  std::vector<std::pair<size_t, size_t>> prod_recs(kp + 1, {0, 0});
  auto product = [&](int j, cudaStream_t q) -> dmrg3s_status {   // w = H v_j (v_j in vcur)
    const size_t r0 = c->prof.recs.size();
    dmrg3s_status r = run_plan(c, heff, Ldata, vcur, ws1, ws2, 1.0, ws2, Rdata, w, q, prec,
                               &hints);
    if (j >= 0) prod_recs[j] = {r0, c->prof.recs.size()};
    return r != DMRG3S_OK ? fail(c, r, "H_eff launch failed") : DMRG3S_OK;
  };
  // Iteration k on stream q with k from the device counter: two Gram-Schmidt
  // passes (the update of the first fused with the dots of the second),
  // v_{k+1} into the basis and vcur, w = H v_{k+1}, k += 1.
  auto body = [&](cudaStream_t q, int j) -> dmrg3s_status {
    launch_lz_dots(V, ldv, 0, w, dch, nchunks, part, kp, q, kdev);
    launch_lz_update_dots(V, ldv, 0, w, dch, nchunks, dcn, part, kp, alpha, part2, q, kdev);
    launch_lz_update(V, ldv, 0, w, dch, nchunks, dcn, part2, kp, nullptr, nrm, q, kdev, nchunks);
    launch_lz_next(w, V, ldv, kdev, vcur, dch, nchunks, dcn, nrm, nchunks, q);
    dmrg3s_status r = product(j, q);
    launch_lz_advance(kdev, q);
    return r;
  };
  if ((s = product(0, st))) return bail(s);
  // Without the profiler, the iteration is captured once into a CUDA graph
  // (every kernel reads k from the device counter) and replayed; with it,
  // the launches are issued directly so that each product is recorded.
  cudaGraphExec_t gexec = nullptr;
  if (!c->prof.on && c->cap) {
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const dmrg3s_status r = body(c->cap, -1);
      ok = cudaStreamEndCapture(c->cap, &graph) == cudaSuccess && r == DMRG3S_OK;
    }
    if (ok && cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) gexec = nullptr;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();   // a failed capture leaves the direct launches
  }
  // the host's reading of iteration k
  auto collect = [&](int k) -> dmrg3s_status {
    if (cudaEventSynchronize(c->ev_lz[k % kLzLag]) != cudaSuccess)
      return fail(c, DMRG3S_ERR_CUDA, "Lanczos step");
    const double* sl = pin + (size_t)(k % kLzLag) * slot;
    int dev_err = 0;
    std::memcpy(&dev_err, sl + (size_t)np * 4, sizeof(int));
    if (dev_err) {
      cudaStreamSynchronize(st);
      cudaStreamSynchronize(c->aux);
      cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
      cudaStreamSynchronize(st);
      return fail(c, DMRG3S_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
    }
    for (int i = 0; i < np; ++i) {
      if (kstop[i] >= 0) continue;
      TridiagOut res;
      std::memcpy(&res, sl + (size_t)i * 4, sizeof(res));
      if (res.nan_seen != 0.0) return fail(c, DMRG3S_ERR_NUMERIC, "NaN in the Lanczos recursion");
      const bool conv = res.resid <= probs[i].tol * std::fmax(1.0, std::fabs(res.theta));
      if (conv || res.beta_last < 1e-14 || k + 1 == probs[i].kmax) {
        kstop[i] = k;
        (*theta)[i] = res.theta;
        (*iters)[i] = k + 1;
        ++nstopped;
      }
    }
    return DMRG3S_OK;
  };
  // The host reads iteration k's results two iterations later, so that the
  // device always has the next iteration queued while the side stream solves
  // the tridiagonal problem.
  constexpr int kLagRead = kLzLag - 1;
  int last = -1;   // the last iteration enqueued
  int next_read = 0;
  for (int k = 0; k < kmax; ++k) {
    if (gexec) {
      if (cudaGraphLaunch(gexec, st) != cudaSuccess)
        s = fail(c, DMRG3S_ERR_CUDA, "Lanczos iteration graph");
    } else {
      s = body(st, k + 1);
    }
    if (s) {
      if (gexec) cudaGraphExecDestroy(gexec);
      return bail(s);
    }
    cudaEventRecord(c->ev_ready, st);
    cudaStreamWaitEvent(c->aux, c->ev_ready, 0);
    launch_lz_tridiag(dcn, np, alpha, beta, kp, k, nrm + (int64_t)(k % kLzLag) * nchunks, y, out,
                      c->aux);
    double* sl = pin + (size_t)(k % kLzLag) * slot;
    cudaMemcpyAsync(sl, out + (size_t)k * np, sizeof(TridiagOut) * np, cudaMemcpyDeviceToHost,
                    c->aux);
    cudaMemcpyAsync(sl + (size_t)np * 4, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->aux);
    cudaEventRecord(c->ev_lz[k % kLzLag], c->aux);
    last = k;
    if (k >= kLagRead) {
      if ((s = collect(next_read++))) break;
      if (nstopped == np) break;
    }
  }
  while (!s && nstopped < np && next_read <= last) s = collect(next_read++);
  if (!s && nstopped < np) s = fail(c, DMRG3S_ERR_CUDA, "Lanczos did not stop");
  if (s) {
    if (gexec) cudaGraphExecDestroy(gexec);
    return bail(s);
  }
  int kmaxstop = 0;
  for (int i = 0; i < np; ++i) kmaxstop = std::max(kmaxstop, kstop[i]);
  for (int j = kmaxstop + 1; j <= kp; ++j)   // the discarded products (direct launches only)
    for (size_t r = prod_recs[j].first; r < prod_recs[j].second; ++r) {
      c->prof.recs[r].flops = 0.0;
      c->prof.recs[r].bytes = 0.0;
    }
  // Ritz vectors x = V y (y written on the side stream), normalised
  cudaEventRecord(c->ev_ready, c->aux);
  cudaStreamWaitEvent(st, c->ev_ready, 0);
  if (cudaMemcpyAsync(dks, kstop.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st) !=
      cudaSuccess) {
    if (gexec) cudaGraphExecDestroy(gexec);
    return bail(fail(c, DMRG3S_ERR_CUDA, "Lanczos tables"));
  }
  launch_lz_ritz(V, ldv, dch, nchunks, dcn, dks, y, kp, w, nrm_x, st);
  launch_lz_normalise(w, X, dch, nchunks, dcn, nrm_x, st);
  if (gexec) {   // its last replays may still run: free it once they are done
    cudaStreamSynchronize(st);
    cudaGraphExecDestroy(gexec);
  }
  if (cudaGetLastError() != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "Lanczos launch failed");
  return DMRG3S_OK;
}

dmrg3s_status lanczos_run(Context* c, const DevicePlan& heff, const double* Ldata,
                          const double* Rdata, double* x, int64_t n, int kmax, double tol,
                          size_t cursor, cudaStream_t st, double* theta, int* iters,
                          dmrg3s_precision prec) {
  std::vector<LzSpec> one(1, LzSpec{0, n, kmax, tol});
  std::vector<double> th;
  std::vector<int> it;
  dmrg3s_status s = lanczos_batch(c, heff, Ldata, Rdata, x, n, one, cursor, st, prec, &th, &it);
  if (s != DMRG3S_OK) return s;
  *theta = th[0];
  *iters = it[0];
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
