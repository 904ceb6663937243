// Library context: device, workspace arena, cached device-resident plans.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "plan.hpp"

namespace dmrg3s {

// Device copy of a plan's task tables.
struct DevicePlan {
  Plan host;
  void* mem = nullptr;      // one allocation holding every table
  GemmTile* g1_tiles = nullptr;
  GemmTask* g1_tasks = nullptr;
  GemmSeg* g1_segs = nullptr;
  CombChunk* c2_chunks = nullptr;
  CombTask* c2_tasks = nullptr;
  CombTerm* c2_terms = nullptr;
  GemmTile* g3_tiles = nullptr;
  GemmTask* g3s_tasks = nullptr;     // split-K stage 3 (tensor-core form)
  // tensor-core tables: units, segments and operand packs of stages 1 and 3,
  // and the packed outputs of stage 2
  TcUnit* g1_units = nullptr;
  int32_t* g1_cta = nullptr;
  TcSeg* g1_tsegs = nullptr;
  PackBlock* g1_packA = nullptr;
  PackBlock* g1_packB = nullptr;
  TcUnit* g3s_units = nullptr;
  int32_t* g3s_cta = nullptr;
  TcSeg* g3s_tsegs = nullptr;
  PackBlock* g3s_packA = nullptr;
  PackBlock* g3s_packB = nullptr;
  PackOut* c2_pack = nullptr;
  GemmTask* g12_tasks = nullptr;     // fused stages 1 + 2 of the tensor-core H_eff
  TcUnit* g12_units = nullptr;
  int32_t* g12_cta = nullptr;
  TcSeg* g12_tsegs = nullptr;
  PackBlock* g12_packA = nullptr;
  PackBlock* g12_packB = nullptr;
  CombChunk* c3r_chunks = nullptr;
  CombTask* c3r_tasks = nullptr;
  CombTerm* c3r_terms = nullptr;
  GemmTask* g3_tasks = nullptr;
  GemmSeg* g3_segs = nullptr;
  ~DevicePlan();
};

// Per-kernel timing with CUDA events recorded on the launching stream around
// every grouped-GEMM and combination launch while profiling is on.
enum ProfKind {
  kProfGemm = 0,        // grouped-GEMM launches
  kProfCombine = 1,     // MPO combination launches
  kProfEig = 2,         // phases of a local update: eigensolver
  kProfExpand = 3,      //   expansion term
  kProfSvd = 4,         //   gather of M~, per-sector SVD, selection, new tensors
  kProfRemainder = 5,   //   S V^dagger (or U S) into the neighbour
  kProfEnv = 6,         //   environment update
  kProfEnergy = 7,      //   energy after truncation
  kProfAuxGemm = 8,     // FP64 grouped GEMMs outside H_eff/expansion/environment:
                        //   the remainder of the truncation, the MPO-entry gradient
  kProfJacobi = 9,      // one Jacobi sweep of the truncation's SVD (all its round launches)
  kProfKinds = 10
};
struct ProfRec {
  int kind;
  cudaEvent_t e0, e1;
  double flops, bytes;
  int64_t launches = 1;   // kernel launches between e0 and e1
};
struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t take() {
    cudaEvent_t e;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  int begin(int kind, double flops, double bytes, cudaStream_t st) {
    ProfRec r{kind, take(), take(), flops, bytes};
    cudaEventRecord(r.e0, st);
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void end(int id, cudaStream_t st) { cudaEventRecord(recs[id].e1, st); }
  void reset() {
    for (auto& r : recs) {
      pool.push_back(r.e0);
      pool.push_back(r.e1);
    }
    recs.clear();
  }
  ~Profiler() {
    reset();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct Context {
  Profiler prof;
  int device = 0;
  char* ws = nullptr;           // workspace arena
  size_t ws_bytes = 0;
  double* pinned = nullptr;     // small pinned host buffer for scalar read-backs (64 doubles)
  int* d_err = nullptr;         // device error word latched by bounded waits (tensor-core kernel)
  uint64_t wait_ns = 1000000000ull;   // limit of every bounded device wait (dmrg3s_set_wait_limit)
  cudaStream_t aux = nullptr;   // side stream: the Lanczos tridiagonal solve beside the next product
  cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
  cudaEvent_t ev_lz[3] = {nullptr, nullptr, nullptr};   // Lanczos results of iterations k mod 3
  cudaStream_t cap = nullptr;   // private stream for capturing the Lanczos iteration graph
  double* pinned_big = nullptr;   // pinned read-back area of the batched Lanczos (grown on demand)
  size_t pinned_big_n = 0;        // its size in doubles
  std::unordered_map<uint64_t, std::unique_ptr<DevicePlan>> plans;
  std::string last_error;
};

// FNV-1a fingerprint builder used as the plan-cache key.
struct Hasher {
  uint64_t h = 1469598103934665603ull;
  void bytes(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
  template <class T>
  void pod(const T& v) { bytes(&v, sizeof(T)); }
  template <class T>
  void vec(const std::vector<T>& v) {
    pod(v.size());
    if (!v.empty()) bytes(v.data(), v.size() * sizeof(T));
  }
  void bond(const Bond& b);
  void site(const SiteLayout& s);
  void env(const EnvLayout& e);
  void mpo(const MpoLayout& w);
};

inline dmrg3s_status fail(Context* c, dmrg3s_status st, const std::string& msg) {
  if (c) c->last_error = msg;
  return st;
}

inline dmrg3s_status use_device(Context* c) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "cudaGetDevice failed");
  if (cur != c->device && cudaSetDevice(c->device) != cudaSuccess)
    return fail(c, DMRG3S_ERR_CUDA, "cudaSetDevice failed");
  return DMRG3S_OK;
}

// Cached plans.  Each returns the device plan for the given structures,
// building and uploading it on first use.
dmrg3s_status heff_plan(Context* c, const EnvLayout& le, const MpoLayout& w, const EnvLayout& re,
                        const SiteLayout& a, const DevicePlan** out);
dmrg3s_status expand_plan(Context* c, int dir, const EnvLayout& e, const MpoLayout& w,
                          const SiteLayout& m, const SiteLayout& P, const FusedBond& f,
                          const DevicePlan** out);
dmrg3s_status env_plan(Context* c, int dir, const EnvLayout& e, const MpoLayout& w,
                       const SiteLayout& a, const EnvLayout& o, const DevicePlan** out);

// Bump allocator over the context workspace: returns an aligned pointer at
// byte offset *cursor and advances it; DMRG3S_ERR_OOM when it does not fit.
inline dmrg3s_status carve(Context* c, size_t* cursor, size_t bytes, void** out) {
  size_t off = (*cursor + 255) / 256 * 256;
  if (off + bytes > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM, "context workspace too small (need " +
                                       std::to_string(off + bytes) + " bytes)");
  *out = c->ws + off;
  *cursor = off + bytes;
  return DMRG3S_OK;
}

// Lanczos with CGS2 for the smallest eigenpair of H_eff (step 1 of Sec. V).
// x: start vector on input, normalised Ritz vector on output (n doubles).
// The workspace from byte offset `cursor` on is used for the Krylov basis.
dmrg3s_status lanczos_run(Context* c, const DevicePlan& heff, const double* Ldata,
                          const double* Rdata, double* x, int64_t n, int kmax, double tol,
                          size_t cursor, cudaStream_t st, double* theta, int* iters,
                          dmrg3s_precision prec = DMRG3S_FP64);

// The same for several independent problems at once: `heff` is a plan whose
// vector operand holds every problem back to back (problem c at elements
// [off, off + n) of X, off a multiple of 32, ldx >= every off + n), so that one
// launch per stage applies all their H_eff.  Each problem keeps its own
// stopping rule (kmax, tol); theta and iters get one entry per problem.
struct LzSpec {
  int64_t off, n;
  int kmax;
  double tol;
};
dmrg3s_status lanczos_batch(Context* c, const DevicePlan& heff, const double* Ldata,
                            const double* Rdata, double* X, int64_t ldx,
                            const std::vector<LzSpec>& probs, size_t cursor, cudaStream_t st,
                            dmrg3s_precision prec, std::vector<double>* theta,
                            std::vector<int>* iters);
// Pinned host area of at least n doubles (c->pinned_big).
dmrg3s_status pinned_reserve(Context* c, size_t n);

// Upload a host plan (allocates the device tables).  Returns CUDA errors.
dmrg3s_status upload_plan(Plan&& host, std::unique_ptr<DevicePlan>* out);

// Enqueue the stages of a plan.  Bases as documented for each plan Kind.
// Tensor-core mode: the stage-1 and stage-3 operands are packed (hi, lo
// parts, tile layout of kernels.hpp) into the workspace:
//   [T1 pairs: ws1][packed T2 (stage-2 output)][g1 A packed][g1 B packed]
//   [g3 A or B packed (the operand that is not T2)][stage-3 partial pairs: ws3]
// (the fused H_eff has no T1 slot, and its stage-1 operands are g12's: the
// coefficient-scaled L blocks and the site tensor)
// (offsets in doubles, each slot 1 KB aligned; a packed operand of n floats
// per part takes n doubles: hi then lo).  A caller that has already packed an
// operand into its slot passes a hint and run_plan skips that pack (the
// Lanczos loop packs L and R once per run).
struct SplitHints {
  bool g1A = false, g1B = false, g3A = false, g3B = false;
  // H_eff only: packed L (stage-1 A) and R (stage-3 B) held outside the
  // workspace (a prepared operator); when set they replace those slots
  const float *g1A_hi = nullptr, *g1A_lo = nullptr, *g3B_hi = nullptr, *g3B_lo = nullptr;
};
struct TcSlots {
  int64_t t2p, a1, b1, x3, p3, end;   // offsets in doubles from the workspace start
};
inline int64_t slot_round(int64_t d) { return (d + 127) / 128 * 128; }   // 1 KB
inline TcSlots tc_slots(const Plan& p) {
  // the fused H_eff never forms T1; its stage-1 operands are g12's
  const TcStage& s1 = p.fused ? p.g12.tc : p.g1.tc;
  TcSlots s;
  s.t2p = p.fused ? 0 : slot_round(p.ws1);
  s.a1 = s.t2p + slot_round(p.nT2p);
  s.b1 = s.a1 + slot_round(s1.nA);
  s.x3 = s.b1 + slot_round(s1.nB);
  const int64_t n3 = p.kind == Kind::Heff ? p.g3s.tc.nB : p.g3s.tc.nA;
  s.p3 = s.x3 + slot_round(p.has_g3 ? n3 : 0);
  s.end = s.p3 + slot_round(p.ws3);
  return s;
}
// Workspace (in doubles) a plan needs in the given precision.
inline int64_t plan_ws_doubles(const Plan& p, dmrg3s_precision prec) {
  return prec == DMRG3S_FP64 ? p.ws1 + p.ws2 : tc_slots(p).end;
}

// `prec` selects the grouped-GEMM kernel of stages 1 and 3 (the combination
// of stage 2 is always FP64).
dmrg3s_status run_plan(Context* c, const DevicePlan& p, const double* g1A, const double* g1B,
                       double* ws1, double* c2out, double c2scale, const double* g3A,
                       const double* g3B, double* g3C, cudaStream_t st,
                       dmrg3s_precision prec = DMRG3S_FP64, const SplitHints* hints = nullptr);

// MPO-entry gradient G (d*d*wl*wr doubles, device, layout of W) of
// <M|H_eff|M> for the given environments; intermediates in the workspace.
dmrg3s_status run_mpo_grad(Context* c, const GradPlan& p, const double* L, const double* M,
                           const double* R, double* G, cudaStream_t st);

}  // namespace dmrg3s
