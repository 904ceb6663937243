// MPO-entry gradient of the DMRG3S energy functional.
//
// <Psi|H|Psi> is linear in every MPO tensor W_i (the network of Sec. II), so
// its derivative with respect to the entries of W_i is the same network with
// W_i taken out:
//   G_i[s', s, bl, br] = sum L_{i-1}[bl](al', al) M_i[s'](al', ar') M_i[s](al, ar)
//                            R_{i+1}[br](ar', ar)
// and, divided by <Psi|Psi>, dE/dtheta = sum_i <G_i, dW_i/dtheta> at fixed
// Psi (Hellmann-Feynman at a stationary state).  The contraction reuses the
// first stage of the H_eff order of Sec. V (T1 = L M), contracts the bra copy
// of M with R on the other side (Y = M R), and finishes with one blockwise
// inner product per entry of G.  FP64 throughout.
#include <cstring>

#include "context.hpp"
#include "dmrg3s.h"
#include "validate.hpp"

namespace dmrg3s {

namespace {

template <class T>
dmrg3s_status put(Context* c, const std::vector<T>& v, T** dev, cudaStream_t st) {
  *dev = nullptr;
  if (v.empty()) return DMRG3S_OK;
  cudaError_t e = cudaMallocAsync((void**)dev, v.size() * sizeof(T), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(*dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "gradient table upload");
  return DMRG3S_OK;
}

dmrg3s_status gemm_stage(Context* c, const GemmStage& g, const double* A, const double* B,
                         double* C, cudaStream_t st) {
  if (g.tiles.empty()) return DMRG3S_OK;
  GemmTile* dt;
  GemmTask* dk;
  GemmSeg* ds;
  dmrg3s_status s;
  if ((s = put(c, g.tiles, &dt, st)) || (s = put(c, g.tasks, &dk, st)) ||
      (s = put(c, g.segs, &ds, st)))
    return s;
  const int id = c->prof.on ? c->prof.begin(kProfAuxGemm, g.flops, g.bytes, st) : -1;
  launch_gemm_f64(g.ta, g.tb, dt, (int)g.tiles.size(), dk, ds, A, B, C, st);
  if (id >= 0) c->prof.end(id, st);
  cudaFreeAsync(dt, st);
  cudaFreeAsync(dk, st);
  if (ds) cudaFreeAsync(ds, st);
  return DMRG3S_OK;
}

}  // namespace

dmrg3s_status run_mpo_grad(Context* c, const GradPlan& p, const double* L, const double* M,
                           const double* R, double* G, cudaStream_t st) {
  if ((size_t)(p.ws1 + p.wsy) * sizeof(double) > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM, "context workspace too small for the gradient intermediates");
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* wsy = ws1 + p.ws1;
  dmrg3s_status s;
  if ((s = gemm_stage(c, p.g1, L, M, ws1, st)) || (s = gemm_stage(c, p.gy, M, R, wsy, st)))
    return s;
  DotTask* dt;
  DotSeg* ds;
  if ((s = put(c, p.tasks, &dt, st)) || (s = put(c, p.segs, &ds, st))) return s;
  launch_dots(dt, (int)p.tasks.size(), ds, ws1, wsy, G, st);
  cudaFreeAsync(dt, st);
  if (ds) cudaFreeAsync(ds, st);
  if (cudaGetLastError() != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "gradient launch");
  return DMRG3S_OK;
}

}  // namespace dmrg3s

using namespace dmrg3s;

extern "C" dmrg3s_status dmrg3s_mpo_grad_site(dmrg3s_ctx ctx, const dmrg3s_env* L,
                                              const dmrg3s_mpo_site* W, const dmrg3s_env* R,
                                              const dmrg3s_site* M, double* G,
                                              dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !L || !W || !R || !M || !G) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  std::string err;
  EnvLayout le, re;
  MpoLayout w;
  SiteLayout m;
  dmrg3s_status st;
  if ((st = make_env(L, &le, &err)) || (st = make_env(R, &re, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(M, &m, &err)))
    return fail(c, st, err);
  if ((st = check_site_mpo(m, w, &err)) ||
      (st = check_env(le, m.left, w.wl, w.tl, "L", &err)) ||
      (st = check_env(re, m.right, w.wr, w.tr, "R", &err)))
    return fail(c, st, err);
  if (!L->data || !R->data || !M->data) return fail(c, DMRG3S_ERR_ARG, "NULL device data pointer");
  GradPlan p;
  if ((st = plan_mpo_grad(le, w, re, m, &p, &err))) return fail(c, st, err);
  if ((st = use_device(c))) return st;
  return run_mpo_grad(c, p, L->data, M->data, R->data, G, reinterpret_cast<cudaStream_t>(stream));
}
