// H_eff application that allocates no device memory.
//
// Some callers cannot call cudaMalloc: real-time or embedded hosts whose
// device memory is fully reserved up front, or frameworks that own the
// allocator and forbid foreign allocations.  For them,
// dmrg3s_apply_heff_noalloc runs the same FP64
// contraction as dmrg3s_apply_heff without a context: the intermediates
// T1 = L A and T2 = W T1 and the task tables live in the fixed-size static
// device arrays below, which every GPU that loads this library holds until
// the process exits.
//
// Host code only sees host-side stand-ins for these arrays, never their
// device addresses; the device addresses are obtained once per device with
// cudaGetSymbolAddress (on the first call made on that device, with that
// device current) and passed to the kernels.
#include <cstring>
#include <mutex>

#include "dmrg3s.h"
#include "kernels.hpp"
#include "plan.hpp"

using namespace dmrg3s;

namespace {

constexpr int64_t kScratchDoubles = DMRG3S_NOALLOC_SCRATCH_DOUBLES;
constexpr int64_t kMaxTiles = 65536, kMaxTasks = 32768, kMaxSegs = 65536;
constexpr int64_t kMaxChunks = 131072, kMaxCombTasks = 32768, kMaxTerms = 131072;

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) GemmTile g_tiles[2][kMaxTiles];
static __device__ __align__(256) GemmTask g_tasks[2][kMaxTasks];
static __device__ __align__(256) GemmSeg g_segs[2][kMaxSegs];
static __device__ __align__(256) CombChunk g_chunks[kMaxChunks];
static __device__ __align__(256) CombTask g_ctasks[kMaxCombTasks];
static __device__ __align__(256) CombTerm g_terms[kMaxTerms];

struct DeviceSymbols {
  bool ready = false;
  double* scratch = nullptr;
  GemmTile* tiles = nullptr;
  GemmTask* tasks = nullptr;
  GemmSeg* segs = nullptr;
  CombChunk* chunks = nullptr;
  CombTask* ctasks = nullptr;
  CombTerm* terms = nullptr;
};

constexpr int kMaxDevices = 64;
DeviceSymbols g_sym[kMaxDevices];
std::mutex g_sym_mutex;

// Device addresses of the static arrays on the current device (set-up on the
// first call per device).
dmrg3s_status symbols(int dev, DeviceSymbols** out) {
  if (dev < 0 || dev >= kMaxDevices) return DMRG3S_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_sym_mutex);
  DeviceSymbols& s = g_sym[dev];
  if (!s.ready) {
    if (cudaGetSymbolAddress((void**)&s.scratch, g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s.tiles, g_tiles) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s.tasks, g_tasks) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s.segs, g_segs) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s.chunks, g_chunks) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s.ctasks, g_ctasks) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s.terms, g_terms) != cudaSuccess)
      return DMRG3S_ERR_CUDA;
    s.ready = true;
  }
  *out = &s;
  return DMRG3S_OK;
}

template <class T>
cudaError_t put(T* dst, const std::vector<T>& v, cudaStream_t st) {
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

}  // namespace

extern "C" dmrg3s_status dmrg3s_apply_heff_noalloc(const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                                   const dmrg3s_env* R, const dmrg3s_site* A,
                                                   dmrg3s_site* HA, dmrg3s_stream stream) {
  if (!L || !W || !R || !A || !HA) return DMRG3S_ERR_ARG;
  std::string err;
  dmrg3s_status st;
  EnvLayout le, re;
  MpoLayout w;
  SiteLayout a, ha;
  if ((st = make_env(L, &le, &err)) || (st = make_env(R, &re, &err)) ||
      (st = make_mpo(W, &w, &err)) || (st = make_site(A, &a, &err)) ||
      (st = make_site(HA, &ha, &err)))
    return st;
  if ((st = check_site_mpo(a, w, &err)) || (st = check_env(le, a.left, w.wl, w.tl, "L", &err)) ||
      (st = check_env(re, a.right, w.wr, w.tr, "R", &err)))
    return st;
  if (!same_bond(a.left, ha.left) || !same_bond(a.right, ha.right) || a.d != ha.d ||
      !same_charges(a.qp, ha.qp))
    return DMRG3S_ERR_SHAPE;
  if (!L->data || !R->data || !A->data || !HA->data) return DMRG3S_ERR_ARG;
  Plan p;
  if ((st = plan_heff(le, w, re, a, &p, &err))) return st;
  // every intermediate and table must fit its static array
  if (p.ws1 + p.ws2 > kScratchDoubles || (int64_t)p.g1.tiles.size() > kMaxTiles ||
      (int64_t)p.g3.tiles.size() > kMaxTiles || (int64_t)p.g1.tasks.size() > kMaxTasks ||
      (int64_t)p.g3.tasks.size() > kMaxTasks || (int64_t)p.g1.segs.size() > kMaxSegs ||
      (int64_t)p.g3.segs.size() > kMaxSegs || (int64_t)p.c2.chunks.size() > kMaxChunks ||
      (int64_t)p.c2.tasks.size() > kMaxCombTasks || (int64_t)p.c2.terms.size() > kMaxTerms)
    return DMRG3S_ERR_LIMIT;
  // an error left pending by earlier work on this thread is not ours to
  // clear, and would be mistaken for a failure of these launches
  if (cudaPeekAtLastError() != cudaSuccess) return DMRG3S_ERR_CUDA;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DMRG3S_ERR_CUDA;
  DeviceSymbols* s = nullptr;
  if ((st = symbols(dev, &s))) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  GemmTile* t1 = s->tiles;
  GemmTile* t3 = s->tiles + kMaxTiles;
  GemmTask* k1 = s->tasks;
  GemmTask* k3 = s->tasks + kMaxTasks;
  GemmSeg* g1 = s->segs;
  GemmSeg* g3 = s->segs + kMaxSegs;
  if (put(t1, p.g1.tiles, cs) || put(k1, p.g1.tasks, cs) || put(g1, p.g1.segs, cs) ||
      put(t3, p.g3.tiles, cs) || put(k3, p.g3.tasks, cs) || put(g3, p.g3.segs, cs) ||
      put(s->chunks, p.c2.chunks, cs) || put(s->ctasks, p.c2.tasks, cs) ||
      put(s->terms, p.c2.terms, cs))
    return DMRG3S_ERR_CUDA;
  // intermediates: every element of T1 and T2 is written before it is read,
  // so the contents left by an earlier call need no clearing
  double* ws1 = s->scratch;
  double* ws2 = s->scratch + p.ws1;
  launch_gemm_f64(p.g1.ta, p.g1.tb, t1, (int)p.g1.tiles.size(), k1, g1, L->data, A->data, ws1, cs);
  launch_combine_f64(s->chunks, (int)p.c2.chunks.size(), s->ctasks, s->terms, ws1, ws2, 1.0, cs);
  launch_gemm_f64(p.g3.ta, p.g3.tb, t3, (int)p.g3.tiles.size(), k3, g3, ws2, R->data, HA->data, cs);
  return cudaGetLastError() == cudaSuccess ? DMRG3S_OK : DMRG3S_ERR_CUDA;
}
