// extern "C" entry points of the contraction part of the C ABI (include/dmrg3s.h).
#include <cstring>
#include <new>

#include "context.hpp"
#include "dmrg3s.h"

using namespace dmrg3s;

namespace dmrg3s {

void Hasher::bond(const Bond& b) {
  pod(b.nsym);
  vec(b.q);
  vec(b.dim);
}
void Hasher::site(const SiteLayout& s) {
  pod(s.nsym);
  pod(s.d);
  vec(s.qp);
  bond(s.left);
  bond(s.right);
}
void Hasher::env(const EnvLayout& e) {
  pod(e.nsym);
  pod(e.w);
  vec(e.t);
  bond(e.bond);
}
void Hasher::mpo(const MpoLayout& w) {
  pod(w.nsym);
  pod(w.d);
  pod(w.wl);
  pod(w.wr);
  vec(w.qp);
  vec(w.tl);
  vec(w.tr);
  vec(w.W);
}

DevicePlan::~DevicePlan() {
  if (mem) cudaFree(mem);
}

namespace {
template <class T>
size_t bytes_of(const std::vector<T>& v) {
  return ((v.size() * sizeof(T)) + 255) / 256 * 256;
}
template <class T>
T* place(char* base, size_t* off, const std::vector<T>& v, std::vector<char>* staging) {
  T* p = reinterpret_cast<T*>(base + *off);
  if (!v.empty()) std::memcpy(staging->data() + *off, v.data(), v.size() * sizeof(T));
  *off += bytes_of(v);
  return v.empty() ? nullptr : p;
}
}  // namespace

dmrg3s_status upload_plan(Plan&& host, std::unique_ptr<DevicePlan>* out) {
  std::unique_ptr<DevicePlan> dp(new (std::nothrow) DevicePlan());
  if (!dp) return DMRG3S_ERR_OOM;
  dp->host = std::move(host);
  const Plan& h = dp->host;
  size_t total = bytes_of(h.g1.tiles) + bytes_of(h.g1.tasks) + bytes_of(h.g1.segs) +
                 bytes_of(h.c2.chunks) + bytes_of(h.c2.tasks) + bytes_of(h.c2.terms) +
                 bytes_of(h.g3.tiles) + bytes_of(h.g3.tasks) + bytes_of(h.g3.segs) +
                 bytes_of(h.g3s.tasks) + bytes_of(h.c3r.chunks) + bytes_of(h.c3r.tasks) +
                 bytes_of(h.c3r.terms) + bytes_of(h.g1.tc.units) + bytes_of(h.g1.tc.segs) +
                 bytes_of(h.g1.tc.packA) + bytes_of(h.g1.tc.packB) + bytes_of(h.g3s.tc.units) +
                 bytes_of(h.g3s.tc.segs) + bytes_of(h.g3s.tc.packA) + bytes_of(h.g3s.tc.packB) +
                 bytes_of(h.c2pack) + bytes_of(h.g12.tasks) + bytes_of(h.g12.tc.units) +
                 bytes_of(h.g12.tc.segs) + bytes_of(h.g12.tc.packA) + bytes_of(h.g12.tc.packB) +
                 bytes_of(h.g1.tc.cta_start) + bytes_of(h.g3s.tc.cta_start) +
                 bytes_of(h.g12.tc.cta_start);
  if (total == 0) total = 256;
  if (cudaMalloc(&dp->mem, total) != cudaSuccess) return DMRG3S_ERR_CUDA;
  std::vector<char> staging(total, 0);
  char* base = static_cast<char*>(dp->mem);
  size_t off = 0;
  dp->g1_tiles = place(base, &off, h.g1.tiles, &staging);
  dp->g1_tasks = place(base, &off, h.g1.tasks, &staging);
  dp->g1_segs = place(base, &off, h.g1.segs, &staging);
  dp->c2_chunks = place(base, &off, h.c2.chunks, &staging);
  dp->c2_tasks = place(base, &off, h.c2.tasks, &staging);
  dp->c2_terms = place(base, &off, h.c2.terms, &staging);
  dp->g3_tiles = place(base, &off, h.g3.tiles, &staging);
  dp->g3_tasks = place(base, &off, h.g3.tasks, &staging);
  dp->g3_segs = place(base, &off, h.g3.segs, &staging);
  dp->g3s_tasks = place(base, &off, h.g3s.tasks, &staging);
  dp->g1_units = place(base, &off, h.g1.tc.units, &staging);
  dp->g1_tsegs = place(base, &off, h.g1.tc.segs, &staging);
  dp->g1_packA = place(base, &off, h.g1.tc.packA, &staging);
  dp->g1_packB = place(base, &off, h.g1.tc.packB, &staging);
  dp->g3s_units = place(base, &off, h.g3s.tc.units, &staging);
  dp->g3s_tsegs = place(base, &off, h.g3s.tc.segs, &staging);
  dp->g3s_packA = place(base, &off, h.g3s.tc.packA, &staging);
  dp->g3s_packB = place(base, &off, h.g3s.tc.packB, &staging);
  dp->c2_pack = place(base, &off, h.c2pack, &staging);
  dp->g12_tasks = place(base, &off, h.g12.tasks, &staging);
  dp->g12_units = place(base, &off, h.g12.tc.units, &staging);
  dp->g12_tsegs = place(base, &off, h.g12.tc.segs, &staging);
  dp->g12_packA = place(base, &off, h.g12.tc.packA, &staging);
  dp->g12_packB = place(base, &off, h.g12.tc.packB, &staging);
  dp->g1_cta = place(base, &off, h.g1.tc.cta_start, &staging);
  dp->g3s_cta = place(base, &off, h.g3s.tc.cta_start, &staging);
  dp->g12_cta = place(base, &off, h.g12.tc.cta_start, &staging);
  dp->c3r_chunks = place(base, &off, h.c3r.chunks, &staging);
  dp->c3r_tasks = place(base, &off, h.c3r.tasks, &staging);
  dp->c3r_terms = place(base, &off, h.c3r.terms, &staging);
  if (cudaMemcpy(dp->mem, staging.data(), total, cudaMemcpyHostToDevice) != cudaSuccess)
    return DMRG3S_ERR_CUDA;
  *out = std::move(dp);
  return DMRG3S_OK;
}

dmrg3s_status run_plan(Context* c, const DevicePlan& p, const double* g1A, const double* g1B,
                       double* ws1, double* c2out, double c2scale, const double* g3A,
                       const double* g3B, double* g3C, cudaStream_t st, dmrg3s_precision prec,
                       const SplitHints* hints) {
  const Plan& h = p.host;
  Profiler& pr = c->prof;
  const int passes = prec == DMRG3S_TF32X3 ? 3 : prec == DMRG3S_TF32 ? 1 : 0;
  if (!passes) {
    if (!h.g1.tiles.empty()) {
      const int id = pr.on ? pr.begin(kProfGemm, h.g1.flops, h.g1.bytes, st) : -1;
      launch_gemm_f64(h.g1.ta, h.g1.tb, p.g1_tiles, (int)h.g1.tiles.size(), p.g1_tasks,
                      p.g1_segs, g1A, g1B, ws1, st);
      if (id >= 0) pr.end(id, st);
    }
    if (!h.c2.chunks.empty()) {
      const int id = pr.on ? pr.begin(kProfCombine, h.c2.flops, h.c2.bytes, st) : -1;
      launch_combine_f64(p.c2_chunks, (int)h.c2.chunks.size(), p.c2_tasks, p.c2_terms, ws1,
                         c2out, c2scale, st);
      if (id >= 0) pr.end(id, st);
    }
    if (h.has_g3 && !h.g3.tiles.empty()) {
      const int id = pr.on ? pr.begin(kProfGemm, h.g3.flops, h.g3.bytes, st) : -1;
      launch_gemm_f64(h.g3.ta, h.g3.tb, p.g3_tiles, (int)h.g3.tiles.size(), p.g3_tasks,
                      p.g3_segs, g3A, g3B, g3C, st);
      if (id >= 0) pr.end(id, st);
    }
    return cudaGetLastError() == cudaSuccess ? DMRG3S_OK : DMRG3S_ERR_CUDA;
  }
  // ---- tensor-core mode: packed (hi, lo) operands
  const TcSlots sl = tc_slots(h);
  double* base = reinterpret_cast<double*>(c->ws);
  auto hi = [&](int64_t slot) { return reinterpret_cast<float*>(base + slot); };
  auto lo = [&](int64_t slot, int64_t n) {
    return passes == 3 ? reinterpret_cast<float*>(base + slot) + n : nullptr;
  };
  const SplitHints none;
  const SplitHints& hn = hints ? *hints : none;
  // the tensor-core stages write double-float pairs (8 bytes per element, in
  // place of the FP64 intermediates), combined on the FP32 pipe
  float2* t1p = reinterpret_cast<float2*>(ws1);
  if (h.fused) {
    // H_eff: stages 1 and 2 in one grouped GEMM over the MPO terms, writing T2
    // packed as the stage-3 operand (T1 is never formed)
    const TcStage& t12 = h.g12.tc;
    if (!hn.g1A) launch_pack(p.g12_packA, (int)t12.packA.size(), t12.tilesA, g1A, hi(sl.a1),
                             lo(sl.a1, t12.nA), st);
    if (!hn.g1B) launch_pack(p.g12_packB, (int)t12.packB.size(), t12.tilesB, g1B, hi(sl.b1),
                             lo(sl.b1, t12.nB), st);
    const float* aH = hn.g1A_hi ? hn.g1A_hi : hi(sl.a1);
    const float* aL = hn.g1A_hi ? hn.g1A_lo : lo(sl.a1, t12.nA);
    if (!t12.units.empty()) {
      const int id = pr.on ? pr.begin(kProfGemm, h.g12.flops, h.g12.bytes, st) : -1;
      launch_gemm_tc(passes, true, p.g12_units, p.g12_cta, (int)t12.cta_start.size() - 1,
                     p.g12_tasks, p.g12_tsegs, aH, aL, hi(sl.b1), lo(sl.b1, t12.nB), hi(sl.t2p),
                     lo(sl.t2p, h.nT2p), c->d_err, c->wait_ns, st);
      if (id >= 0) pr.end(id, st);
    }
  } else {
    const TcStage& t1 = h.g1.tc;
    if (!hn.g1A) launch_pack(p.g1_packA, (int)t1.packA.size(), t1.tilesA, g1A, hi(sl.a1),
                             lo(sl.a1, t1.nA), st);
    if (!hn.g1B) launch_pack(p.g1_packB, (int)t1.packB.size(), t1.tilesB, g1B, hi(sl.b1),
                             lo(sl.b1, t1.nB), st);
    if (!t1.units.empty()) {
      const int id = pr.on ? pr.begin(kProfGemm, h.g1.flops, h.g1.bytes, st) : -1;
      launch_gemm_tc(passes, false, p.g1_units, p.g1_cta, (int)t1.cta_start.size() - 1,
                     p.g1_tasks, p.g1_tsegs,
                     hi(sl.a1), lo(sl.a1, t1.nA), hi(sl.b1), lo(sl.b1, t1.nB),
                     reinterpret_cast<float*>(t1p), nullptr, c->d_err, c->wait_ns, st);
      if (id >= 0) pr.end(id, st);
    }
  }
  if (!h.has_g3) {
    if (!h.c2.chunks.empty()) {
      const int id = pr.on ? pr.begin(kProfCombine, h.c2.flops, h.c2.bytes, st) : -1;
      launch_combine_pairs_f64(p.c2_chunks, (int)h.c2.chunks.size(), p.c2_tasks, p.c2_terms,
                               t1p, c2out, c2scale, st);
      if (id >= 0) pr.end(id, st);
    }
    return cudaGetLastError() == cudaSuccess ? DMRG3S_OK : DMRG3S_ERR_CUDA;
  }
  // stage 2 writes T2 packed as the stage-3 operand it feeds
  if (!h.fused && !h.c2pack.empty()) {
    const int id = pr.on ? pr.begin(kProfCombine, h.c2.flops, h.c2.bytes, st) : -1;
    launch_combine_pairs_pack(p.c2_pack, (int)h.c2pack.size(), h.tilesT2, p.c2_tasks, p.c2_terms,
                              t1p, hi(sl.t2p), lo(sl.t2p, h.nT2p), c2scale, st);
    if (id >= 0) pr.end(id, st);
  }
  // stage 3: T2 is A for H_eff, B for the environment updates; the other
  // operand is packed into slot x3 (unless the caller already did)
  const TcStage& t3 = h.g3s.tc;
  const bool t2_is_a = h.kind == Kind::Heff;
  const float *a3h, *a3l, *b3h, *b3l;
  if (t2_is_a) {
    a3h = hi(sl.t2p);
    a3l = lo(sl.t2p, h.nT2p);
    if (!hn.g3B) launch_pack(p.g3s_packB, (int)t3.packB.size(), t3.tilesB, g3B, hi(sl.x3),
                             lo(sl.x3, t3.nB), st);
    b3h = hn.g3B_hi ? hn.g3B_hi : hi(sl.x3);
    b3l = hn.g3B_hi ? hn.g3B_lo : lo(sl.x3, t3.nB);
  } else {
    if (!hn.g3A) launch_pack(p.g3s_packA, (int)t3.packA.size(), t3.tilesA, g3A, hi(sl.x3),
                             lo(sl.x3, t3.nA), st);
    a3h = hi(sl.x3);
    a3l = lo(sl.x3, t3.nA);
    b3h = hi(sl.t2p);
    b3l = lo(sl.t2p, h.nT2p);
  }
  // split-K: one unit per (tile, K-segment) into double-float partials, then
  // a fixed-order sum
  float2* part = reinterpret_cast<float2*>(base + sl.p3);
  if (!t3.units.empty()) {
    const int id = pr.on ? pr.begin(kProfGemm, h.g3s.flops, h.g3s.bytes, st) : -1;
    launch_gemm_tc(passes, false, p.g3s_units, p.g3s_cta, (int)t3.cta_start.size() - 1,
                   p.g3s_tasks, p.g3s_tsegs,
                   a3h, a3l, b3h, b3l, reinterpret_cast<float*>(part), nullptr, c->d_err,
                   c->wait_ns, st);
    if (id >= 0) pr.end(id, st);
  }
  if (!h.c3r.chunks.empty()) {
    const int id = pr.on ? pr.begin(kProfCombine, 0.0, 0.0, st) : -1;
    launch_combine_pairs_f64(p.c3r_chunks, (int)h.c3r.chunks.size(), p.c3r_tasks, p.c3r_terms,
                             part, g3C, 1.0, st);
    if (id >= 0) pr.end(id, st);
  }
  return cudaGetLastError() == cudaSuccess ? DMRG3S_OK : DMRG3S_ERR_CUDA;
}

}  // namespace dmrg3s

namespace {

// Fetch a cached plan or build and upload one.
template <class Build>
dmrg3s_status get_plan(Context* c, uint64_t key, Build build, const DevicePlan** out) {
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    *out = it->second.get();
    return DMRG3S_OK;
  }
  Plan p;
  std::string err;
  dmrg3s_status st = build(&p, &err);
  if (st != DMRG3S_OK) return fail(c, st, err);
  std::unique_ptr<DevicePlan> dp;
  st = upload_plan(std::move(p), &dp);
  if (st != DMRG3S_OK) return fail(c, st, "uploading a contraction plan failed");
  *out = dp.get();
  c->plans[key] = std::move(dp);
  return DMRG3S_OK;
}

}  // namespace

namespace dmrg3s {
dmrg3s_status heff_plan(Context* c, const EnvLayout& le, const MpoLayout& w, const EnvLayout& re,
                        const SiteLayout& a, const DevicePlan** out) {
  Hasher h;
  h.pod((int)Kind::Heff);
  h.env(le);
  h.mpo(w);
  h.env(re);
  h.site(a);
  return get_plan(c, h.h, [&](Plan* pl, std::string* e) { return plan_heff(le, w, re, a, pl, e); },
                  out);
}

dmrg3s_status expand_plan(Context* c, int dir, const EnvLayout& e, const MpoLayout& w,
                          const SiteLayout& m, const SiteLayout& pl, const FusedBond& f,
                          const DevicePlan** out) {
  Hasher h;
  h.pod(dir == 1 ? (int)Kind::ExpandLR : (int)Kind::ExpandRL);
  h.env(e);
  h.mpo(w);
  h.site(m);
  return get_plan(
      c, h.h,
      [&](Plan* pn, std::string* er) {
        return dir == 1 ? plan_expand_lr(e, w, m, pl, f, pn, er)
                        : plan_expand_rl(e, w, m, pl, f, pn, er);
      },
      out);
}

dmrg3s_status env_plan(Context* c, int dir, const EnvLayout& e, const MpoLayout& w,
                       const SiteLayout& a, const EnvLayout& o, const DevicePlan** out) {
  Hasher h;
  h.pod(dir == 1 ? (int)Kind::EnvLR : (int)Kind::EnvRL);
  h.env(e);
  h.mpo(w);
  h.site(a);
  return get_plan(
      c, h.h,
      [&](Plan* pn, std::string* er) {
        return dir == 1 ? plan_env_lr(e, w, a, o, pn, er) : plan_env_rl(e, w, a, o, pn, er);
      },
      out);
}
}  // namespace dmrg3s

namespace {

dmrg3s_status check_ws(Context* c, const Plan& p, dmrg3s_precision prec) {
  const size_t need = (size_t)plan_ws_doubles(p, prec) * sizeof(double);
  if (need > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM,
                "context workspace too small: need " + std::to_string(need) + " bytes");
  return DMRG3S_OK;
}

dmrg3s_status prec_ok(Context* c, dmrg3s_precision prec) {
  if (prec == DMRG3S_FP64 || prec == DMRG3S_TF32X3 || prec == DMRG3S_TF32) return DMRG3S_OK;
  return fail(c, DMRG3S_ERR_ARG, "unknown precision");
}

}  // namespace

extern "C" {

dmrg3s_status dmrg3s_create(dmrg3s_ctx* ctx, int device, size_t workspace_bytes) {
  if (!ctx) return DMRG3S_ERR_ARG;
  *ctx = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DMRG3S_ERR_CUDA;
  Context* c = new (std::nothrow) Context();
  if (!c) return DMRG3S_ERR_OOM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return DMRG3S_ERR_CUDA;
  }
  c->ws_bytes = workspace_bytes ? workspace_bytes : (size_t)256 << 20;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) == cudaSuccess)
    set_plan_ctas(nsm);
  if (cudaMalloc(&c->ws, c->ws_bytes) != cudaSuccess) {
    delete c;
    return DMRG3S_ERR_CUDA;
  }
  // keep freed stream-ordered allocations in the pool (no release at every sync)
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return DMRG3S_ERR_CUDA;
  }
  if (cudaMallocHost(&c->pinned, 64 * sizeof(double)) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return DMRG3S_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_lz[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_lz[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_lz[2], cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFreeHost(c->pinned);
    cudaFree(c->ws);
    delete c;
    return DMRG3S_ERR_CUDA;
  }
  *ctx = reinterpret_cast<dmrg3s_ctx>(c);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_destroy(dmrg3s_ctx ctx) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c) return DMRG3S_ERR_ARG;
  use_device(c);
  cudaDeviceSynchronize();
  c->plans.clear();
  if (c->ws) cudaFree(c->ws);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->d_err) cudaFree(c->d_err);
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  for (cudaEvent_t e : c->ev_lz)
    if (e) cudaEventDestroy(e);
  if (c->pinned_big) cudaFreeHost(c->pinned_big);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
  return DMRG3S_OK;
}

const char* dmrg3s_status_string(dmrg3s_status s) {
  switch (s) {
    case DMRG3S_OK: return "ok";
    case DMRG3S_ERR_ARG: return "invalid argument";
    case DMRG3S_ERR_SHAPE: return "inconsistent shapes";
    case DMRG3S_ERR_QN: return "inconsistent charges";
    case DMRG3S_ERR_OOM: return "out of memory";
    case DMRG3S_ERR_CUDA: return "CUDA error";
    case DMRG3S_ERR_NOT_CONVERGED: return "not converged";
    case DMRG3S_ERR_BREAKDOWN: return "Lanczos breakdown";
    case DMRG3S_ERR_TIMEOUT: return "device wait timed out";
    case DMRG3S_ERR_NUMERIC: return "NaN or Inf";
    case DMRG3S_ERR_UNSUPPORTED: return "unsupported";
    case DMRG3S_ERR_LIMIT: return "exceeds a fixed static capacity";
  }
  return "unknown status";
}

const char* dmrg3s_last_error(dmrg3s_ctx ctx) {
  Context* c = reinterpret_cast<Context*>(ctx);
  return c ? c->last_error.c_str() : "no context";
}

dmrg3s_status dmrg3s_sync(dmrg3s_ctx ctx, dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c) return DMRG3S_ERR_ARG;
  dmrg3s_status st = use_device(c);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int flag = 0;
  if (cudaMemcpyAsync(&c->pinned[0], c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(c, DMRG3S_ERR_CUDA, "synchronisation failed");
  std::memcpy(&flag, &c->pinned[0], sizeof(int));
  if (flag) {
    cudaMemsetAsync(c->d_err, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return fail(c, DMRG3S_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
  }
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_set_wait_limit(dmrg3s_ctx ctx, double seconds) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c) return DMRG3S_ERR_ARG;
  if (!(seconds >= 0.0) || seconds > 1e6) return fail(c, DMRG3S_ERR_ARG, "wait limit");
  c->wait_ns = (uint64_t)(seconds * 1e9);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_profile(dmrg3s_ctx ctx, int32_t enable) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c) return DMRG3S_ERR_ARG;
  c->prof.reset();
  c->prof.on = enable != 0;
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_profile_read(dmrg3s_ctx ctx, int32_t kernel, dmrg3s_kernel_stats* out) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !out || kernel < 0 || kernel >= kProfKinds) return DMRG3S_ERR_ARG;
  out->launches = 0;
  out->ms = out->flops = out->bytes = 0.0;
  for (const ProfRec& r : c->prof.recs) {
    if (r.kind != kernel) continue;
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "profile events");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    out->launches += r.launches;
    out->ms += ms;
    out->flops += r.flops;
    out->bytes += r.bytes;
  }
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_launch_count(int64_t* n) {
  if (!n) return DMRG3S_ERR_ARG;
  *n = launch_count();
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_site_size(const dmrg3s_site* M, int64_t* nelem) {
  if (!nelem) return DMRG3S_ERR_ARG;
  SiteLayout s;
  std::string err;
  dmrg3s_status st = make_site(M, &s, &err);
  if (st != DMRG3S_OK) return st;
  *nelem = s.size;
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_heff_cost(const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                               const dmrg3s_env* R, const dmrg3s_site* A, double* flops,
                               double* bytes) {
  if (!L || !W || !R || !A || !flops) return DMRG3S_ERR_ARG;
  std::string err;
  EnvLayout le, re;
  MpoLayout w;
  SiteLayout a;
  dmrg3s_status st;
  if ((st = make_env(L, &le, &err)) || (st = make_env(R, &re, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(A, &a, &err)))
    return st;
  if ((st = check_site_mpo(a, w, &err)) || (st = check_env(le, a.left, w.wl, w.tl, "L", &err)) ||
      (st = check_env(re, a.right, w.wr, w.tr, "R", &err)))
    return st;
  Plan p;
  if ((st = plan_heff(le, w, re, a, &p, &err))) return st;
  *flops = p.flops();
  if (bytes) *bytes = p.g1.bytes + p.c2.bytes + p.g3.bytes;
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_env_size(const dmrg3s_env* E, int64_t* nelem) {
  if (!nelem) return DMRG3S_ERR_ARG;
  EnvLayout e;
  std::string err;
  dmrg3s_status st = make_env(E, &e, &err);
  if (st != DMRG3S_OK) return st;
  *nelem = e.size;
  return DMRG3S_OK;
}

static void write_table(const std::vector<Block>& blocks, int64_t* nblocks, int64_t* table) {
  *nblocks = (int64_t)blocks.size();
  if (!table) return;
  for (size_t n = 0; n < blocks.size(); ++n) {
    const Block& b = blocks[n];
    int64_t* row = table + 6 * n;
    row[0] = b.a;
    row[1] = b.b;
    row[2] = b.c;
    row[3] = b.off;
    row[4] = b.rows;
    row[5] = b.cols;
  }
}

dmrg3s_status dmrg3s_site_blocks(const dmrg3s_site* M, int64_t* nblocks, int64_t* table) {
  if (!nblocks) return DMRG3S_ERR_ARG;
  SiteLayout s;
  std::string err;
  dmrg3s_status st = make_site(M, &s, &err);
  if (st != DMRG3S_OK) return st;
  write_table(s.blocks, nblocks, table);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_env_blocks(const dmrg3s_env* E, int64_t* nblocks, int64_t* table) {
  if (!nblocks) return DMRG3S_ERR_ARG;
  EnvLayout e;
  std::string err;
  dmrg3s_status st = make_env(E, &e, &err);
  if (st != DMRG3S_OK) return st;
  write_table(e.blocks, nblocks, table);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_expanded_bond(int32_t nsym, const dmrg3s_bond* bond, int32_t w,
                                   const int32_t* t, int32_t include_base, int32_t* nsec,
                                   int32_t* q, int64_t* dim) {
  if (!nsec || w < 1 || (nsym > 0 && !t)) return DMRG3S_ERR_ARG;
  Bond b;
  std::string err;
  dmrg3s_status st = make_bond(nsym, bond, &b, &err);
  if (st != DMRG3S_OK) return st;
  std::vector<Charge> tc(w, Charge{});
  for (int i = 0; i < w; ++i)
    for (int k = 0; k < nsym; ++k) tc[i][k] = t[(size_t)i * nsym + k];
  FusedBond f;
  st = fuse_bond(b, w, tc, include_base != 0, &f);
  if (st != DMRG3S_OK) return st;
  *nsec = f.bond.nsec();
  if (q && nsym > 0)
    for (int i = 0; i < f.bond.nsec(); ++i)
      for (int k = 0; k < nsym; ++k) q[(size_t)i * nsym + k] = f.bond.q[i][k];
  if (dim)
    for (int i = 0; i < f.bond.nsec(); ++i) dim[i] = f.bond.dim[i];
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_apply_heff(dmrg3s_ctx ctx, const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                const dmrg3s_env* R, const dmrg3s_site* A, dmrg3s_site* HA,
                                dmrg3s_precision prec, dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !L || !W || !R || !A || !HA) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  dmrg3s_status st = prec_ok(c, prec);
  if (st != DMRG3S_OK) return st;
  std::string err;
  EnvLayout le, re;
  MpoLayout w;
  SiteLayout a, ha;
  if ((st = make_env(L, &le, &err)) || (st = make_env(R, &re, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(A, &a, &err)) ||
      (st = make_site(HA, &ha, &err)))
    return fail(c, st, err);
  if ((st = check_site_mpo(a, w, &err)) ||
      (st = check_env(le, a.left, w.wl, w.tl, "L", &err)) ||
      (st = check_env(re, a.right, w.wr, w.tr, "R", &err)))
    return fail(c, st, err);
  if (!same_bond(a.left, ha.left) || !same_bond(a.right, ha.right) || a.d != ha.d ||
      !same_charges(a.qp, ha.qp))
    return fail(c, DMRG3S_ERR_SHAPE, "HA must have the structure of A");
  if (!L->data || !R->data || !A->data || !HA->data)
    return fail(c, DMRG3S_ERR_ARG, "NULL device data pointer");
  const DevicePlan* p = nullptr;
  st = heff_plan(c, le, w, re, a, &p);
  if (st != DMRG3S_OK) return st;
  if ((st = check_ws(c, p->host, prec)) || (st = use_device(c))) return st;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + p->host.ws1;
  st = run_plan(c, *p, L->data, A->data, ws1, ws2, 1.0, ws2, R->data, HA->data,
                reinterpret_cast<cudaStream_t>(stream), prec);
  return st == DMRG3S_OK ? st : fail(c, st, "kernel launch failed");
}

dmrg3s_status dmrg3s_expand(dmrg3s_ctx ctx, int32_t dir, const dmrg3s_env* env,
                            const dmrg3s_mpo_site* W, const dmrg3s_site* M, double alpha,
                            dmrg3s_site* P, dmrg3s_precision prec, dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !env || !W || !M || !P) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  if (dir != 1 && dir != -1) return fail(c, DMRG3S_ERR_ARG, "dir must be +1 or -1");
  dmrg3s_status st = prec_ok(c, prec);
  if (st != DMRG3S_OK) return st;
  std::string err;
  EnvLayout e;
  MpoLayout w;
  SiteLayout m, pl;
  if ((st = make_env(env, &e, &err)) || (st = make_mpo(W, &w, &err)) ||
      (st = make_site(M, &m, &err)) || (st = make_site(P, &pl, &err)))
    return fail(c, st, err);
  if ((st = check_site_mpo(m, w, &err))) return fail(c, st, err);
  if (dir == 1) {
    if ((st = check_env(e, m.left, w.wl, w.tl, "env (L)", &err))) return fail(c, st, err);
  } else {
    if ((st = check_env(e, m.right, w.wr, w.tr, "env (R)", &err))) return fail(c, st, err);
  }
  FusedBond f;
  fuse_bond(dir == 1 ? m.right : m.left, dir == 1 ? w.wr : w.wl, dir == 1 ? w.tr : w.tl, false,
            &f);
  const Bond& keep = dir == 1 ? m.left : m.right;
  const Bond& pkeep = dir == 1 ? pl.left : pl.right;
  const Bond& pfused = dir == 1 ? pl.right : pl.left;
  if (!same_bond(keep, pkeep) || !same_bond(f.bond, pfused) || pl.d != m.d ||
      !same_charges(pl.qp, m.qp))
    return fail(c, DMRG3S_ERR_SHAPE, "P does not have the expanded structure of M");
  if (!env->data || !M->data || !P->data) return fail(c, DMRG3S_ERR_ARG, "NULL device data");
  const DevicePlan* p = nullptr;
  st = expand_plan(c, dir, e, w, m, pl, f, &p);
  if (st != DMRG3S_OK) return st;
  if ((st = check_ws(c, p->host, prec)) || (st = use_device(c))) return st;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  const double* g1A = dir == 1 ? env->data : M->data;
  const double* g1B = dir == 1 ? M->data : env->data;
  st = run_plan(c, *p, g1A, g1B, ws1, P->data, alpha, nullptr, nullptr, nullptr,
                reinterpret_cast<cudaStream_t>(stream), prec);
  return st == DMRG3S_OK ? st : fail(c, st, "kernel launch failed");
}

dmrg3s_status dmrg3s_update_env(dmrg3s_ctx ctx, int32_t dir, const dmrg3s_env* env,
                                const dmrg3s_mpo_site* W, const dmrg3s_site* A, dmrg3s_env* out,
                                dmrg3s_precision prec, dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !env || !W || !A || !out) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  if (dir != 1 && dir != -1) return fail(c, DMRG3S_ERR_ARG, "dir must be +1 or -1");
  dmrg3s_status st = prec_ok(c, prec);
  if (st != DMRG3S_OK) return st;
  std::string err;
  EnvLayout e, o;
  MpoLayout w;
  SiteLayout a;
  if ((st = make_env(env, &e, &err)) || (st = make_env(out, &o, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(A, &a, &err)))
    return fail(c, st, err);
  if ((st = check_site_mpo(a, w, &err))) return fail(c, st, err);
  if (dir == 1) {
    if ((st = check_env(e, a.left, w.wl, w.tl, "env (L_{i-1})", &err)) ||
        (st = check_env(o, a.right, w.wr, w.tr, "out (L_i)", &err)))
      return fail(c, st, err);
  } else {
    if ((st = check_env(e, a.right, w.wr, w.tr, "env (R_{i+1})", &err)) ||
        (st = check_env(o, a.left, w.wl, w.tl, "out (R_i)", &err)))
      return fail(c, st, err);
  }
  if (!env->data || !A->data || !out->data) return fail(c, DMRG3S_ERR_ARG, "NULL device data");
  const DevicePlan* p = nullptr;
  st = env_plan(c, dir, e, w, a, o, &p);
  if (st != DMRG3S_OK) return st;
  if ((st = check_ws(c, p->host, prec)) || (st = use_device(c))) return st;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + p->host.ws1;
  const double* g1A = dir == 1 ? env->data : A->data;
  const double* g1B = dir == 1 ? A->data : env->data;
  st = run_plan(c, *p, g1A, g1B, ws1, ws2, 1.0, A->data, ws2, out->data,
                reinterpret_cast<cudaStream_t>(stream), prec);
  return st == DMRG3S_OK ? st : fail(c, st, "kernel launch failed");
}

}  // extern "C"
