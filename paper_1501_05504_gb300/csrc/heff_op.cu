// Prepared H_eff operator: the left-hand side of the local eigenproblem
// (Eq. es-iter, Sec. V) for fixed environments, applied many times.
//
// A Lanczos run applies H_eff = L_{i-1} W_i . R_{i+1} to a new vector in
// every iteration while L, W and R stay fixed.  The handle plans the
// contraction once and, in the tensor-core modes, packs L (as the
// coefficient-scaled blocks of the fused stages 1 + 2) and R (stage-3
// operand) once into device memory it owns, so that each application only
// packs the vector and runs the block products.
#include <new>

#include "context.hpp"
#include "dmrg3s.h"

using namespace dmrg3s;

namespace dmrg3s {
struct HeffOp {
  Context* c = nullptr;
  const DevicePlan* plan = nullptr;
  dmrg3s_precision prec = DMRG3S_FP64;
  const double* L = nullptr;   // the caller's environments (FP64 mode reads them at every apply)
  const double* R = nullptr;
  float* packL = nullptr;      // tensor-core modes: packed copies (hi then lo)
  float* packR = nullptr;
  int64_t nA = 0;              // elements of A and HA
};
}  // namespace dmrg3s

extern "C" {

dmrg3s_status dmrg3s_heff_create(dmrg3s_ctx ctx, const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                 const dmrg3s_env* R, const dmrg3s_site* A,
                                 dmrg3s_precision prec, dmrg3s_heff* out, dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !L || !W || !R || !A || !out) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (prec != DMRG3S_FP64 && prec != DMRG3S_TF32X3 && prec != DMRG3S_TF32)
    return fail(c, DMRG3S_ERR_ARG, "unknown precision");
  std::string err;
  EnvLayout le, re;
  MpoLayout w;
  SiteLayout a;
  dmrg3s_status st;
  if ((st = make_env(L, &le, &err)) || (st = make_env(R, &re, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(A, &a, &err)))
    return fail(c, st, err);
  if ((st = check_site_mpo(a, w, &err)) || (st = check_env(le, a.left, w.wl, w.tl, "L", &err)) ||
      (st = check_env(re, a.right, w.wr, w.tr, "R", &err)))
    return fail(c, st, err);
  if (!L->data || !R->data) return fail(c, DMRG3S_ERR_ARG, "NULL device data");
  if ((st = use_device(c))) return st;
  const DevicePlan* p = nullptr;
  if ((st = heff_plan(c, le, w, re, a, &p))) return st;
  if ((size_t)plan_ws_doubles(p->host, prec) * sizeof(double) > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM, "context workspace too small for H_eff");
  HeffOp* h = new (std::nothrow) HeffOp();
  if (!h) return fail(c, DMRG3S_ERR_OOM, "H_eff handle");
  h->c = c;
  h->plan = p;
  h->prec = prec;
  h->L = L->data;
  h->R = R->data;
  h->nA = a.size;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (prec != DMRG3S_FP64) {
    const Plan& hp = p->host;
    const TcStage& t1 = hp.g12.tc;
    const TcStage& t3 = hp.g3s.tc;
    const bool x3 = prec == DMRG3S_TF32X3;
    if (cudaMalloc(&h->packL, sizeof(float) * (size_t)std::max<int64_t>(t1.nA, 1) * 2) !=
            cudaSuccess ||
        cudaMalloc(&h->packR, sizeof(float) * (size_t)std::max<int64_t>(t3.nB, 1) * 2) !=
            cudaSuccess) {
      if (h->packL) cudaFree(h->packL);
      delete h;
      return fail(c, DMRG3S_ERR_CUDA, "H_eff handle: packed environments");
    }
    launch_pack(p->g12_packA, (int)t1.packA.size(), t1.tilesA, L->data, h->packL,
                x3 ? h->packL + t1.nA : nullptr, s);
    launch_pack(p->g3s_packB, (int)t3.packB.size(), t3.tilesB, R->data, h->packR,
                x3 ? h->packR + t3.nB : nullptr, s);
    if (cudaGetLastError() != cudaSuccess) {
      cudaFree(h->packL);
      cudaFree(h->packR);
      delete h;
      return fail(c, DMRG3S_ERR_CUDA, "H_eff handle: packing launch");
    }
  }
  *out = reinterpret_cast<dmrg3s_heff>(h);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_heff_apply(dmrg3s_heff op, const double* A, double* HA,
                                dmrg3s_stream stream) {
  HeffOp* h = reinterpret_cast<HeffOp*>(op);
  if (!h) return DMRG3S_ERR_ARG;
  Context* c = h->c;
  if (!A || !HA) return fail(c, DMRG3S_ERR_ARG, "NULL device data");
  dmrg3s_status st;
  if ((st = use_device(c))) return st;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + h->plan->host.ws1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SplitHints hints;
  const SplitHints* hp = nullptr;
  if (h->prec != DMRG3S_FP64) {
    const Plan& pl = h->plan->host;
    const bool x3 = h->prec == DMRG3S_TF32X3;
    hints.g1A = true;
    hints.g3B = true;
    hints.g1A_hi = h->packL;
    hints.g1A_lo = x3 ? h->packL + pl.g12.tc.nA : nullptr;
    hints.g3B_hi = h->packR;
    hints.g3B_lo = x3 ? h->packR + pl.g3s.tc.nB : nullptr;
    hp = &hints;
  }
  st = run_plan(c, *h->plan, h->L, A, ws1, ws2, 1.0, ws2, h->R, HA, s, h->prec, hp);
  return st == DMRG3S_OK ? DMRG3S_OK : fail(c, st, "H_eff launch failed");
}

dmrg3s_status dmrg3s_heff_destroy(dmrg3s_heff op) {
  HeffOp* h = reinterpret_cast<HeffOp*>(op);
  if (!h) return DMRG3S_ERR_ARG;
  use_device(h->c);
  if (h->packL || h->packR) cudaDeviceSynchronize();
  if (h->packL) cudaFree(h->packL);
  if (h->packR) cudaFree(h->packR);
  delete h;
  return DMRG3S_OK;
}

}  // extern "C"
