// DMRG3S state (library-owned MPS + environments), the local update of Sec. V
// of arXiv:1501.05504 and the sweep driver with the adaptive mixing factor of
// Sec. VI.
//
// Local update, left-to-right, at site i (right-to-left is the mirror image):
//   1. Lanczos for the smallest eigenpair of H_eff (Eq. es-iter)        [eig.cu]
//   2. expansion term alpha P_i = alpha L_{i-1} M_i W_i (Eq. subexp-ourt) [plan]
//   3. M~ = [M* P] per charge sector of the expanded right bond; the neighbour
//      is padded with zero rows (never materialised: the zero rows only meet
//      the P columns, so step 5 multiplies with the M* part only)
//   4. FP64 SVD of every sector (cuSOLVER gesvd, sectors concurrently on
//      several streams; or QR, then one-sided Jacobi on R^T in this library's
//      kernels, all sectors in each launch [svd.cu]) and global truncation
//      to m_max states: A~ = U
//   5. B~_{i+1} = (S V^dagger)[:, M part] . B_{i+1}                     [grouped GEMM]
//   6. L_i = L_{i-1} A~^dagger W_i A~                                   [plan]
//   7. E_f = <B~|H_eff(i+1)|B~> / <B~|B~> (Rayleigh quotient after truncation)
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>
#include <tuple>

#include "context.hpp"
#include "dmrg3s.h"
#include "svd.hpp"
#include "validate.hpp"
#include "vecops.hpp"

namespace dmrg3s {

namespace {

struct DevSite {
  SiteLayout lay;
  double* data = nullptr;
};
struct DevEnv {
  EnvLayout lay;
  double* data = nullptr;
  bool valid = false;
};

}  // namespace

using SvdWorker = SvdLane;
constexpr int kSvdWorkers = 8;      // default number of concurrent SVD lanes

// Lanes of a new state: DMRG3S_SVD_STREAMS (1..16) when set, else the default.
// A truncation uses about one lane per four charge sectors, at least four
// (one large sector then runs beside the rest) and at most the state's lanes:
// measured on GB300, four lanes suit the 14 sectors of an m=512 XXZ update
// (more add contention), eight the many mid-size sectors of the Hubbard chain.
int svd_lanes() {
  const char* e = std::getenv("DMRG3S_SVD_STREAMS");
  if (!e) return kSvdWorkers;
  const int v = std::atoi(e);
  return v < 1 ? 1 : (v > 16 ? 16 : v);
}

struct State {
  Context* c = nullptr;
  int n = 0;
  std::vector<MpoLayout> W;
  std::vector<DevSite> M;
  std::vector<DevEnv> Lenv;   // Lenv[i]: sites < i, on M[i].left, channels W[i].tl
  std::vector<DevEnv> Renv;   // Renv[i]: sites > i, on M[i].right, channels W[i].tr
  int centre = 0;
  double e_in = 0.0;
  std::vector<SvdWorker> svd;
  cudaEvent_t svd_in = nullptr;
};

namespace {

dmrg3s_status cuda_ok(Context* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DMRG3S_OK;
  return fail(c, DMRG3S_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

dmrg3s_status dalloc(Context* c, double** p, int64_t n, cudaStream_t st) {
  *p = nullptr;
  if (n <= 0) n = 1;
  return cuda_ok(c, cudaMallocAsync((void**)p, (size_t)n * sizeof(double), st), "cudaMallocAsync");
}

void dfree(double* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// Stream-ordered device buffers of one call, freed on `st` on every exit path.
// Work of other streams that uses them is joined into `st` before the call
// can return (svd_sectors, svd_jacobi), so the frees are ordered after it.
struct Scratch {
  Context* c;
  cudaStream_t st;
  std::vector<double*> bufs;
  Scratch(Context* c_, cudaStream_t s) : c(c_), st(s) {}
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    for (double* p : bufs)
      if (p) cudaFreeAsync(p, st);
  }
  dmrg3s_status get(double** p, int64_t n) {
    dmrg3s_status s = dalloc(c, p, n, st);
    if (!s) bufs.push_back(*p);
    return s;
  }
  // frees p now (stream ordered); p must come from get()
  void drop(double* p) {
    for (double*& q : bufs)
      if (q == p && q) {
        cudaFreeAsync(q, st);
        q = nullptr;
      }
  }
  // hands p to the caller, who frees it
  double* keep(double* p) {
    for (double*& q : bufs)
      if (q == p) q = nullptr;
    return p;
  }
};

template <class T>
dmrg3s_status upload(Context* c, const std::vector<T>& v, T** dev, cudaStream_t st) {
  *dev = nullptr;
  if (v.empty()) return DMRG3S_OK;
  cudaError_t e = cudaMallocAsync((void**)dev, v.size() * sizeof(T), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(*dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  return cuda_ok(c, e, "table upload");
}

// Run a host-built grouped GEMM stage (tables uploaded for this call only).
dmrg3s_status run_gemm(Context* c, const GemmStage& g, const double* A, int64_t nA, const double* B,
                       int64_t nB, double* C, int64_t nC, cudaStream_t st) {
  if (g.tiles.empty()) return DMRG3S_OK;
  std::string err;
  if (!gemm_ok(g.ta, g.tb, g.tasks, g.segs, nA, nB, nC, &err))
    return fail(c, DMRG3S_ERR_SHAPE, "internal planning error: " + err);
  GemmTile* dt;
  GemmTask* dk;
  GemmSeg* ds;
  dmrg3s_status s;
  if ((s = upload(c, g.tiles, &dt, st)) || (s = upload(c, g.tasks, &dk, st)) ||
      (s = upload(c, g.segs, &ds, st)))
    return s;
  const int id = c->prof.on ? c->prof.begin(kProfAuxGemm, g.flops, g.bytes, st) : -1;
  launch_gemm_f64(g.ta, g.tb, dt, (int)g.tiles.size(), dk, ds, A, B, C, st);
  if (id >= 0) c->prof.end(id, st);
  cudaFreeAsync(dt, st);
  cudaFreeAsync(dk, st);
  if (ds) cudaFreeAsync(ds, st);
  return cuda_ok(c, cudaGetLastError(), "grouped GEMM");
}

dmrg3s_status run_copies(Context* c, const std::vector<CopyTask>& t, const double* src, int64_t nsrc,
                         double* dst, int64_t ndst, const double* scale, int64_t nscale,
                         cudaStream_t st) {
  if (t.empty()) return DMRG3S_OK;
  std::string err;
  if (!copies_ok(t, nsrc, ndst, nscale, &err))
    return fail(c, DMRG3S_ERR_SHAPE, "internal planning error: " + err);
  CopyTask* dt;
  dmrg3s_status s = upload(c, t, &dt, st);
  if (s) return s;
  launch_copy_blocks(dt, (int)t.size(), src, dst, scale, st);
  cudaFreeAsync(dt, st);
  return cuda_ok(c, cudaGetLastError(), "block copy");
}

CopyTask copy_task(int64_t off_s, int64_t ld_s, int64_t off_d, int64_t ld_d, int64_t rows,
                   int64_t cols, bool trans, int rs = -1, int cs = -1) {
  CopyTask t{};
  t.off_s = off_s;
  t.off_d = off_d;
  t.ld_s = (int32_t)ld_s;
  t.ld_d = (int32_t)ld_d;
  t.rows = (int32_t)rows;
  t.cols = (int32_t)cols;
  t.trans = trans ? 1 : 0;
  t.rs = rs;
  t.cs = cs;
  return t;
}

// <x, y> on the host (synchronises the stream)
dmrg3s_status dot_host(Context* c, const double* x, const double* y, int64_t n, cudaStream_t st,
                       double* out) {
  double *part, *h;
  dmrg3s_status s;
  if ((s = dalloc(c, &part, kRedBlocks, st))) return s;
  if ((s = dalloc(c, &h, 1, st))) {
    dfree(part, st);
    return s;
  }
  launch_multidot(x, 0, 1, y, n, part, h, nullptr, st);
  cudaMemcpyAsync(c->pinned, h, sizeof(double), cudaMemcpyDeviceToHost, st);
  dfree(part, st);
  dfree(h, st);
  if ((s = cuda_ok(c, cudaStreamSynchronize(st), "dot"))) return s;
  *out = c->pinned[0];
  return DMRG3S_OK;
}

// One step of the environment recursion of Sec. II with the current tensor
// of site i: dir = +1 turns the left environment `src` of site i into that of
// site i + 1, dir = -1 the right environment of site i into that of site
// i - 1.  The result is freshly allocated (stream ordered).
dmrg3s_status env_step(State& S, int i, int dir, const EnvLayout& src_lay, const double* src,
                       EnvLayout* out_lay, double** out, cudaStream_t st) {
  Context* c = S.c;
  const MpoLayout& w = S.W[i];
  const DevSite& a = S.M[i];
  make_env_from(a.lay.nsym, dir == 1 ? w.wr : w.wl, dir == 1 ? w.tr : w.tl,
                dir == 1 ? a.lay.right : a.lay.left, out_lay);
  const DevicePlan* p;
  dmrg3s_status s = env_plan(c, dir, src_lay, w, a.lay, *out_lay, &p);
  if (s) return s;
  if ((size_t)(p->host.ws1 + p->host.ws2) * sizeof(double) > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM, "context workspace too small for the environment update");
  if ((s = dalloc(c, out, out_lay->size, st))) return s;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + p->host.ws1;
  const double* g1A = dir == 1 ? src : a.data;
  const double* g1B = dir == 1 ? a.data : src;
  if ((s = run_plan(c, *p, g1A, g1B, ws1, ws2, 1.0, a.data, ws2, *out, st))) {
    dfree(*out, st);
    *out = nullptr;
    return fail(c, s, "environment update launch");
  }
  return DMRG3S_OK;
}

dmrg3s_status build_env(State& S, int i, int dir, cudaStream_t st) {
  DevEnv& src = dir == 1 ? S.Lenv[i] : S.Renv[i];
  if (!src.valid)
    return fail(S.c, DMRG3S_ERR_ARG, "environment recursion from an invalid environment");
  DevEnv& dst = dir == 1 ? S.Lenv[i + 1] : S.Renv[i - 1];
  EnvLayout ol;
  double* nd;
  dmrg3s_status s = env_step(S, i, dir, src.lay, src.data, &ol, &nd, st);
  if (s) return s;
  dfree(dst.data, st);
  dst.data = nd;
  dst.lay = ol;
  dst.valid = true;
  return DMRG3S_OK;
}

// Rayleigh quotient <x|H_eff(i)|x>/<x|x> at site i with the current environments.
dmrg3s_status rayleigh(State& S, int i, const double* x, cudaStream_t st, double* e) {
  Context* c = S.c;
  const DevicePlan* p;
  dmrg3s_status s = heff_plan(c, S.Lenv[i].lay, S.W[i], S.Renv[i].lay, S.M[i].lay, &p);
  if (s) return s;
  if ((size_t)(p->host.ws1 + p->host.ws2) * sizeof(double) > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM, "context workspace too small for H_eff");
  const int64_t n = S.M[i].lay.size;
  Scratch sc(c, st);
  double* hx;
  if ((s = sc.get(&hx, n))) return s;
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + p->host.ws1;
  if ((s = run_plan(c, *p, S.Lenv[i].data, x, ws1, ws2, 1.0, ws2, S.Renv[i].data, hx, st))) return s;
  double num = 0.0, den = 0.0;
  if ((s = dot_host(c, x, hx, n, st, &num)) || (s = dot_host(c, x, x, n, st, &den))) return s;
  *e = den > 0.0 ? num / den : 0.0;
  return DMRG3S_OK;
}

struct Opts {
  int m_max = 64;
  int kmax = 40;
  double tol = 1e-10;       // the caller's Lanczos tolerance (lanczos_tol below applies the floor)
  double eps = 1e-12;
  bool optimise = true;
  dmrg3s_precision prec = DMRG3S_FP64;   // arithmetic of the eigensolver's H_eff products
  dmrg3s_svd_method svd = DMRG3S_SVD_GESVD;
};

// The Lanczos tolerance of a local update: the caller's, but not below the
// accuracy of the products (3xTF32 H_eff ~2e-7 relative, TF32 ~1e-3): below
// it the recursion only resolves the products' rounding.
inline double lanczos_tol(const Opts& o) {
  if (o.prec == DMRG3S_TF32X3) return std::max(o.tol, 3e-7);
  if (o.prec == DMRG3S_TF32) return std::max(o.tol, 3e-4);
  return o.tol;
}

struct Info {
  double lambda = 0.0, e_f = 0.0, discarded = 0.0;
  int iters = 0, new_dim = 0;
  bool svd_fallback = false;
  int svd_sweeps = 0;
};

// One sector of M~ for the SVD: a (rows x cols) row-major matrix.
struct Sector {
  Charge q;
  int64_t rows = 0, cols = 0, base = 0;   // base = size of the M* part (cols for L->R, rows for R->L)
  bool tall = true;                       // rows >= cols: X is factorised, else X^T
  int64_t m = 0, n = 0, r = 0;            // factorised matrix m x n (m >= n), r = n
  int64_t off = 0;                        // offset of the matrix in the X buffer
  int64_t offU = 0, offVT = 0, offS = 0;  // U (m x r), VT (r x n), S (r) in the output buffers
  int keep = 0;
  int jbase = -1;                         // old bond sector of the M* part, -1 if none
  // The kept basis (left vectors for L->R, right vectors for R->L) is the
  // small side n of the factorised matrix: gesvd then forms VT only (no U),
  // and the remainder S V^T (or U S) is the projection of X onto the kept
  // vectors, one GEMM.
  bool vt_only = false;
};

// FP64 SVD X_tall = U S VT of every sector (cuSOLVER gesvd; U only where
// the kept basis is the large side),
// spread over the worker streams, largest sectors first; `st` waits for all.
dmrg3s_status svd_sectors(State& S, const std::vector<Sector>& secs, double* X, double* F,
                          double* Sv, int* info, cudaStream_t st) {
  Context* c = S.c;
  if (secs.empty()) return DMRG3S_OK;
  size_t dmax = 1, hmax = 1;
  for (const Sector& sc : secs) {
    size_t wd = 0, wh = 0;
    if (cusolverDnXgesvd_bufferSize(S.svd[0].h, S.svd[0].p, sc.vt_only ? 'N' : 'S', 'S', sc.m, sc.n,
                                    CUDA_R_64F, nullptr, sc.m, CUDA_R_64F, nullptr, CUDA_R_64F,
                                    nullptr, sc.m, CUDA_R_64F, nullptr, sc.r, CUDA_R_64F, &wd,
                                    &wh) != CUSOLVER_STATUS_SUCCESS)
      return fail(c, DMRG3S_ERR_CUDA, "gesvd buffer size");
    dmax = std::max(dmax, wd);
    hmax = std::max(hmax, wh);
  }
  for (SvdWorker& w : S.svd) {
    if (w.dbytes < dmax) {
      if (w.dwork) cudaFree(w.dwork);
      w.dwork = nullptr;
      w.dbytes = 0;
      if (cudaMalloc(&w.dwork, dmax) != cudaSuccess)
        return fail(c, DMRG3S_ERR_CUDA, "SVD workspace");
      w.dbytes = dmax;
    }
    if (w.hwork.size() < hmax) w.hwork.resize(hmax);
  }
  // greedy assignment by cost m n^2, largest first
  std::vector<int> order(secs.size());
  for (size_t k = 0; k < secs.size(); ++k) order[k] = (int)k;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)secs[a].m * secs[a].n * secs[a].n > (double)secs[b].m * secs[b].n * secs[b].n;
  });
  const int lanes = (int)S.svd.size();
  int nw = (int)secs.size() / 4;
  if (nw < 4) nw = 4;
  if (nw > lanes) nw = lanes;
  std::vector<std::vector<int>> jobs(nw);
  std::vector<double> load(nw, 0.0);
  for (int k : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    jobs[w].push_back(k);
    load[w] += (double)secs[k].m * secs[k].n * secs[k].n + 1e5;
  }
  if (cudaEventRecord(S.svd_in, st) != cudaSuccess) return fail(c, DMRG3S_ERR_CUDA, "SVD event");
  std::vector<int> bad(nw, 0);
  auto run = [&](int w) {
    SvdWorker& wk = S.svd[w];
    cudaSetDevice(c->device);
    cudaStreamWaitEvent(wk.s, S.svd_in, 0);
    cusolverDnSetStream(wk.h, wk.s);
    for (int k : jobs[w]) {
      const Sector& sc = secs[k];
      if (cusolverDnXgesvd(wk.h, wk.p, sc.vt_only ? 'N' : 'S', 'S', sc.m, sc.n, CUDA_R_64F,
                           X + sc.off, sc.m, CUDA_R_64F, Sv + sc.offS, CUDA_R_64F,
                           sc.vt_only ? nullptr : F + sc.offU, sc.m, CUDA_R_64F,
                           F + sc.offVT, sc.r, CUDA_R_64F, wk.dwork, wk.dbytes, wk.hwork.data(),
                           wk.hwork.size(), info + k) != CUSOLVER_STATUS_SUCCESS)
        bad[w] = 1;
    }
    cudaEventRecord(wk.ev, wk.s);
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; ++w)
    if (!jobs[w].empty()) th.emplace_back(run, w);
  if (!jobs[0].empty()) run(0);
  for (auto& t : th) t.join();
  // `st` waits for every lane that ran, also when one of them failed: the
  // caller frees the buffers the lanes use on `st`
  bool any_bad = false;
  for (int w = 0; w < nw; ++w) {
    any_bad = any_bad || bad[w];
    if (!jobs[w].empty()) cudaStreamWaitEvent(st, S.svd[w].ev, 0);
  }
  if (any_bad) return fail(c, DMRG3S_ERR_CUDA, "gesvd");
  return cuda_ok(c, cudaGetLastError(), "SVD launch");
}

// Host side of steps 3 and 4 of one update, left-to-right (dir = +1) or
// right-to-left (dir = -1): the charge sectors of M~ = [M* P] (or [M*; P]),
// the copy tasks that gather M* and P into them, and the placement of every
// sector's SVD factors.
struct Trunc {
  std::vector<Sector> secs;
  std::vector<CopyTask> gather_m, gather_p;
  int64_t xoff = 0, foff = 0, soff = 0;   // elements of X (all sectors), of U / VT, of S
  bool any_proj = false;                  // a copy of X is needed (projected remainders,
                                          // or the restart of a Jacobi SVD)
  // after the selection (truncate_centre): the new bond and the remainder
  Bond nbnd;
  std::vector<int> sec_of_new;            // sector of every sector of the new bond
  std::vector<int64_t> rem_off;           // S V^dagger (or U S) block of every new sector
  int64_t rem_size = 0;
  double* rem = nullptr;                  // owned: freed by update_neighbour
  dmrg3s_svd_method method = DMRG3S_SVD_GESVD;   // the factorisation used (AUTO resolved)
};

// Smaller side of the largest sector from which DMRG3S_SVD_AUTO takes the
// Jacobi SVD.
constexpr int64_t kSvdAutoJacobiN = 192;

void prepare_truncation(const SiteLayout& ml, int dir, bool expand, const FusedBond& fp,
                        const SiteLayout& pl, dmrg3s_svd_method svd, dmrg3s_precision prec,
                        Trunc* t) {
  const Bond& old = dir == 1 ? ml.right : ml.left;
  // Sector k of M~ is a rows x cols matrix X (rows: (s, a_l) for L->R, the
  // expanded left states for R->L).  It is gathered column-major in the tall
  // orientation m >= n that the FP64 SVD routine needs: X itself when
  // rows >= cols, X^T otherwise.
  std::vector<Charge> charges;
  for (int k = 0; k < old.nsec(); ++k) charges.push_back(old.q[k]);
  if (expand)
    for (int k = 0; k < fp.bond.nsec(); ++k) charges.push_back(fp.bond.q[k]);
  std::sort(charges.begin(), charges.end());
  charges.erase(std::unique(charges.begin(), charges.end()), charges.end());
  const Bond& keepb = dir == 1 ? ml.left : ml.right;   // the bond that is not expanded
  std::vector<Sector>& secs = t->secs;
  std::vector<CopyTask>& gather_m = t->gather_m;
  std::vector<CopyTask>& gather_p = t->gather_p;
  secs.clear();
  gather_m.clear();
  gather_p.clear();
  int64_t xoff = 0;
  // task placing a row-major block (rb x cb) at (row0, col0) of sector sc's X
  auto place = [](const Sector& sc, int64_t src_off, int64_t rb, int64_t cb, int64_t row0,
                  int64_t col0) {
    if (sc.tall)   // column-major X (ld rows): write X^T rows = block columns
      return copy_task(src_off, cb, sc.off + col0 * sc.rows + row0, sc.rows, cb, rb, true);
    return copy_task(src_off, cb, sc.off + row0 * sc.cols + col0, sc.cols, rb, cb, false);
  };
  for (const Charge& q : charges) {
    Sector sc;
    sc.q = q;
    sc.jbase = old.find(q);
    if (ml.nsym == 0) sc.jbase = 0;
    const int kp = expand ? (ml.nsym ? fp.bond.find(q) : 0) : -1;
    const int64_t pwidth = kp >= 0 ? fp.bond.dim[kp] : 0;
    sc.base = sc.jbase >= 0 ? old.dim[sc.jbase] : 0;
    const int64_t exp_dim = sc.base + pwidth;
    // the other dimension: sum over physical states of the matching sector of keepb
    int64_t other = 0;
    std::vector<std::pair<int, int64_t>> parts;   // (s, offset along the other dimension)
    for (int ss = 0; ss < ml.d; ++ss) {
      Charge qo = dir == 1 ? sub(q, ml.qp[ss]) : add(q, ml.qp[ss]);
      const int io = ml.nsym ? keepb.find(qo) : 0;
      if (io < 0) continue;
      parts.push_back({ss, other});
      other += keepb.dim[io];
    }
    if (other == 0 || exp_dim == 0) continue;
    sc.rows = dir == 1 ? other : exp_dim;
    sc.cols = dir == 1 ? exp_dim : other;
    sc.tall = sc.rows >= sc.cols;
    sc.m = sc.tall ? sc.rows : sc.cols;
    sc.n = sc.tall ? sc.cols : sc.rows;
    sc.r = sc.n;
    sc.vt_only = dir == 1 ? !sc.tall : sc.tall;
    sc.off = xoff;
    xoff += sc.rows * sc.cols;
    for (auto& pr : parts) {
      const int ss = pr.first;
      const int64_t o2 = pr.second;
      Charge qo = dir == 1 ? sub(q, ml.qp[ss]) : add(q, ml.qp[ss]);
      const int io = ml.nsym ? keepb.find(qo) : 0;
      const int64_t dio = keepb.dim[io];
      if (sc.jbase >= 0) {
        // M* block (ss, io, jbase) for L->R; (ss, jbase, io) for R->L
        const int bi = dir == 1 ? ml.block_of(ss, io) : ml.block_of(ss, sc.jbase);
        if (bi >= 0) {
          const Block& bk = ml.blocks[bi];
          const bool match = dir == 1 ? bk.c == sc.jbase : bk.c == io;
          if (match) {
            if (dir == 1)
              gather_m.push_back(place(sc, bk.off, dio, sc.base, o2, 0));
            else
              gather_m.push_back(place(sc, bk.off, sc.base, dio, 0, o2));
          }
        }
      }
      if (kp >= 0) {
        const int bi = dir == 1 ? pl.block_of(ss, io) : pl.block_of(ss, kp);
        if (bi >= 0) {
          const Block& bk = pl.blocks[bi];
          const bool match = dir == 1 ? bk.c == kp : bk.c == io;
          if (match) {
            if (dir == 1)
              gather_p.push_back(place(sc, bk.off, dio, pwidth, o2, sc.base));
            else
              gather_p.push_back(place(sc, bk.off, pwidth, dio, sc.base, o2));
          }
        }
      }
    }
    secs.push_back(sc);
  }
  t->xoff = xoff;
  // X_tall = U S VT with U (m x r, ld m), VT (r x n, ld r), r = n
  int64_t foff = 0, soff = 0;
  for (Sector& sc : secs) {
    sc.offU = foff;
    if (!sc.vt_only) foff += sc.m * sc.r;
    sc.offVT = foff;
    foff += sc.r * sc.n;
    sc.offS = soff;
    soff += sc.r;
  }
  t->foff = foff;
  t->soff = soff;
  if (svd == DMRG3S_SVD_AUTO) {
    // the Jacobi rounds win on large sectors of FP64 updates; after a 3xTF32
    // or TF32 eigensolver the kept vector carries ~1e-7 noise, whose cluster of
    // small singular values takes the Jacobi sweeps longer than gesvd
    int64_t nmax = 0;
    for (const Sector& sc : secs) nmax = std::max(nmax, sc.n);
    svd = prec == DMRG3S_FP64 && nmax >= kSvdAutoJacobiN ? DMRG3S_SVD_JACOBI : DMRG3S_SVD_GESVD;
  }
  t->method = svd;
  bool any_proj = svd == DMRG3S_SVD_JACOBI;
  for (const Sector& sc : secs) any_proj = any_proj || (sc.vt_only && sc.base > 0);
  t->any_proj = any_proj;
}

// Step 4 for the sectors `secs` (offsets into X, F, Sv): FP64 SVD of every
// sector, the singular values read back into hs (host), every sector's
// convergence checked.  X0 holds a copy of X (needed by the Jacobi method,
// which restores X from it and falls back to gesvd when a sector's sweeps do
// not converge).  dinfo: room for one int per sector.  Synchronises `st`.
dmrg3s_status svd_all(State& S, dmrg3s_svd_method method, const std::vector<Sector>& secs,
                      double* X, const double* X0, int64_t nX, double* F, double* Sv, int* dinfo,
                      int64_t nS, std::vector<double>* hs, bool* fallback, int* sweeps,
                      cudaStream_t st) {
  Context* c = S.c;
  dmrg3s_status s;
  hs->assign(std::max<int64_t>(nS, 1), 0.0);
  std::vector<int> hinfo(secs.size() + 1, 0);
  if (method == DMRG3S_SVD_JACOBI) {
    std::vector<SvdJob> jobs(secs.size());
    for (size_t k = 0; k < secs.size(); ++k) {
      const Sector& sc = secs[k];
      jobs[k].m = sc.m;
      jobs[k].n = sc.n;
      jobs[k].offA = sc.off;
      jobs[k].offS = sc.offS;
      jobs[k].offVT = sc.offVT;
      jobs[k].offU = sc.vt_only ? -1 : sc.offU;
    }
    int nw = (int)secs.size() / 4;
    nw = std::min(std::max(nw, 4), (int)S.svd.size());
    if ((s = svd_jacobi(c, S.svd, nw, jobs, X, Sv, F, F, hinfo.data(), st, nullptr, sweeps)))
      return s;
    bool conv = true;
    for (size_t k = 0; k < secs.size(); ++k) conv = conv && hinfo[k] == 0;
    if (!conv) {   // redo the SVD with gesvd on the restored X
      *fallback = true;
      if ((s = cuda_ok(c, cudaMemcpyAsync(X, X0, (size_t)nX * sizeof(double),
                                          cudaMemcpyDeviceToDevice, st), "copy of M~")) ||
          (s = svd_sectors(S, secs, X, F, Sv, dinfo, st)) ||
          (s = cuda_ok(c, cudaMemcpyAsync(hinfo.data(), dinfo, secs.size() * sizeof(int),
                                          cudaMemcpyDeviceToHost, st), "SVD info")))
        return s;
    }
  } else if ((s = svd_sectors(S, secs, X, F, Sv, dinfo, st)) ||
             (s = cuda_ok(c, cudaMemcpyAsync(hinfo.data(), dinfo, secs.size() * sizeof(int),
                                             cudaMemcpyDeviceToHost, st), "SVD info"))) {
    return s;
  }
  if ((s = cuda_ok(c, cudaMemcpyAsync(hs->data(), Sv, nS * sizeof(double), cudaMemcpyDeviceToHost,
                                      st), "singular values")) ||
      (s = cuda_ok(c, cudaStreamSynchronize(st), "SVD")))
    return s;
  for (size_t k = 0; k < secs.size(); ++k)
    if (hinfo[k] != 0) return fail(c, DMRG3S_ERR_NUMERIC, "SVD did not converge in a sector");
  return DMRG3S_OK;
}

// Selection of step 4 and the new tensors: the states kept over all sectors
// (the largest singular values, at most m_max, above eps times the largest),
// the new centre tensor A~ (L->R) or B~ (R->L) in place of the old one, and
// the remainder S V^dagger (or U S) of every kept sector into t.rem.  F / Sv
// / X0 hold this update's SVD factors and copy of M~ (offsets of t.secs), hs
// its singular values on the host.
dmrg3s_status truncate_centre(State& S, int dir, const Opts& o, Trunc& t, const double* F,
                              const double* Sv, const double* X0, const double* hs, Info* info,
                              cudaStream_t st) {
  Context* c = S.c;
  DevSite& m = S.M[S.centre];
  const SiteLayout& ml = m.lay;
  const Bond& keepb = dir == 1 ? ml.left : ml.right;   // the bond that is not expanded
  std::vector<Sector>& secs = t.secs;
  dmrg3s_status s;
  Scratch scr(c, st);
  // global selection: order by (-s, sector, index), cut at eps * s_max and m_max
  std::vector<std::tuple<double, int, int>> cand;
  double smax = 0.0, total = 0.0;
  for (size_t k = 0; k < secs.size(); ++k)
    for (int64_t j = 0; j < secs[k].r; ++j) {
      const double v = hs[secs[k].offS + j];
      if (!(v == v)) return fail(c, DMRG3S_ERR_NUMERIC, "NaN singular value");
      cand.emplace_back(-v, (int)k, (int)j);
      smax = std::max(smax, v);
      total += v * v;
    }
  std::sort(cand.begin(), cand.end());
  double kept_w = 0.0;
  int nkeep = 0;
  for (auto& t : cand) {
    const double v = -std::get<0>(t);
    if (!(v > o.eps * smax) || nkeep >= o.m_max) break;
    secs[std::get<1>(t)].keep++;
    kept_w += v * v;
    ++nkeep;
  }
  info->discarded = total - kept_w;
  info->new_dim = nkeep;
  if (nkeep == 0) return fail(c, DMRG3S_ERR_NUMERIC, "truncation kept no state");
  // ---- new bond
  Bond& nbnd = t.nbnd;
  nbnd = Bond();
  nbnd.nsym = ml.nsym;
  std::vector<int>& sec_of_new = t.sec_of_new;
  sec_of_new.clear();
  for (size_t k = 0; k < secs.size(); ++k)
    if (secs[k].keep > 0) {
      nbnd.q.push_back(secs[k].q);
      nbnd.dim.push_back(secs[k].keep);
      sec_of_new.push_back((int)k);
    }
  nbnd.off.assign(nbnd.dim.size() + 1, 0);
  for (size_t k = 0; k < nbnd.dim.size(); ++k) nbnd.off[k + 1] = nbnd.off[k] + nbnd.dim[k];
  nbnd.total = nbnd.off.back();
  if (nbnd.nsym == 0) nbnd.q.assign(1, Charge{});
  // ---- new centre tensor A~ (L->R) or B~ (R->L), and the remainder SV / US.
  // With X = U_X S V_X^T: tall sectors have U_X = U, V_X = VT^T; wide ones
  // (X^T was factorised) have U_X = VT^T, V_X = U.
  SiteLayout nl;
  if (dir == 1)
    make_site_from(ml.nsym, ml.d, ml.qp, ml.left, nbnd, &nl);
  else
    make_site_from(ml.nsym, ml.d, ml.qp, nbnd, ml.right, &nl);
  // copy tasks reading U_X[row0 + a, c] (dst a x c) and V_X[col0 + a, c] (dst c x a, or a x c)
  auto ux = [](const Sector& sc, int64_t row0, int64_t dst, int64_t ldd, int64_t na, int64_t nc,
               int cs) {   // dst (na x nc): U_X[row0 + a, c] * S[c]
    if (sc.tall) return copy_task(sc.offU + row0, sc.m, dst, ldd, na, nc, true, -1, cs);
    return copy_task(sc.offVT + row0 * sc.r, sc.r, dst, ldd, na, nc, false, -1, cs);
  };
  auto vxt = [](const Sector& sc, int64_t col0, int64_t dst, int64_t ldd, int64_t nc, int64_t na,
                int rs) {  // dst (nc x na): V_X[col0 + a, c] * S[c]
    if (sc.tall) return copy_task(sc.offVT + col0 * sc.r, sc.r, dst, ldd, nc, na, true, rs, -1);
    return copy_task(sc.offU + col0, sc.m, dst, ldd, nc, na, false, rs, -1);
  };
  std::vector<CopyTask> cp_new, cp_rem;
  GemmStage proj_lr, proj_rl;   // remainder by projection (vt_only sectors)
  proj_lr.ta = Trans::T;
  proj_lr.tb = Trans::N;
  proj_rl.ta = Trans::T;
  proj_rl.tb = Trans::N;
  t.rem_off.assign(nbnd.nsec(), 0);
  std::vector<int64_t>& rem_off = t.rem_off;
  int64_t rem_size = 0;
  for (int kn = 0; kn < nbnd.nsec(); ++kn) {
    const Sector& sc = secs[sec_of_new[kn]];
    const int64_t nk = sc.keep;
    rem_off[kn] = rem_size;
    rem_size += nk * sc.base;
    int64_t o2 = 0;
    for (int ss = 0; ss < ml.d; ++ss) {
      Charge qo = dir == 1 ? sub(sc.q, ml.qp[ss]) : add(sc.q, ml.qp[ss]);
      const int io = ml.nsym ? keepb.find(qo) : 0;
      if (io < 0) continue;
      const int64_t dio = keepb.dim[io];
      const int bi = dir == 1 ? nl.block_of(ss, io) : nl.block_of(ss, kn);
      if (bi >= 0) {
        const Block& bk = nl.blocks[bi];
        if (dir == 1)   // A~ block (dio x nk) = U_X[o2 + a, c]
          cp_new.push_back(ux(sc, o2, bk.off, bk.cols, dio, nk, -1));
        else            // B~ block (nk x dio) = V_X[o2 + a, c]^T
          cp_new.push_back(vxt(sc, o2, bk.off, bk.cols, nk, dio, -1));
      }
      o2 += dio;
    }
    if (sc.base > 0 && sc.vt_only) {
      // L->R (X^T factorised): SV[c, j] = sum_a VT[c, a] X[a, j], X row-major (rows x cols)
      // R->L (X factorised):   US[i, c] = sum_a X[i, a] VT[c, a], X column-major (rows x cols)
      // Both read VT[c, a] at offVT + a r + c, i.e. K x nk row-major with ld r.
      GemmSeg q{};
      q.scale = 1.0;
      q.K = (int32_t)sc.n;
      if (dir == 1) {     // C (nk x base) = VT^T^T . X: A = VT (K x nk, ld r), B = X (K x base, ld cols)
        q.offA = sc.offVT;
        q.lda = (int32_t)sc.r;
        q.offB = sc.off;
        q.ldb = (int32_t)sc.cols;
        proj_lr.add(rem_off[kn], (int)sc.base, (int)nk, (int)sc.base, {q});
      } else {            // C (base x nk) = X^T^T . VT^T: A = X (K x base, ld rows), B = VT (K x nk, ld r)
        q.offA = sc.off;
        q.lda = (int32_t)sc.rows;
        q.offB = sc.offVT;
        q.ldb = (int32_t)sc.r;
        proj_rl.add(rem_off[kn], (int)nk, (int)sc.base, (int)nk, {q});
      }
    } else if (sc.base > 0) {
      if (dir == 1)     // SV (nk x base) = S[c] V_X[col, c]^T
        cp_rem.push_back(vxt(sc, 0, rem_off[kn], sc.base, nk, sc.base, (int)sc.offS));
      else              // US (base x nk) = U_X[row, c] S[c]
        cp_rem.push_back(ux(sc, 0, rem_off[kn], nk, sc.base, nk, (int)sc.offS));
    }
  }
  double *ndata, *rem;
  if ((s = scr.get(&ndata, nl.size)) || (s = scr.get(&rem, rem_size))) return s;
  cudaMemsetAsync(ndata, 0, (size_t)std::max<int64_t>(nl.size, 1) * sizeof(double), st);
  if ((s = run_copies(c, cp_new, F, t.foff, ndata, nl.size, Sv, t.soff, st)) ||
      (s = run_copies(c, cp_rem, F, t.foff, rem, rem_size, Sv, t.soff, st)))
    return s;
  if (dir == 1) {
    if ((s = run_gemm(c, proj_lr, F, t.foff, X0, t.xoff, rem, rem_size, st))) return s;
  } else {
    if ((s = run_gemm(c, proj_rl, X0, t.xoff, F, t.foff, rem, rem_size, st))) return s;
  }
  const SiteLayout nlay = nl;
  dfree(m.data, st);
  m.lay = nlay;
  m.data = scr.keep(ndata);
  t.rem = scr.keep(rem);
  t.rem_size = rem_size;
  return DMRG3S_OK;
}

// Step 5: the remainder S V^dagger (L->R) or U S (R->L) of t multiplied into
// the neighbour site nb, which replaces it (the grouped FP64 GEMM of one
// launch over its blocks); frees t.rem.
dmrg3s_status update_neighbour(State& S, int dir, int nb, Trunc& t, cudaStream_t st) {
  Context* c = S.c;
  const Bond& nbnd = t.nbnd;
  const std::vector<Sector>& secs = t.secs;
  const std::vector<int>& sec_of_new = t.sec_of_new;
  const std::vector<int64_t>& rem_off = t.rem_off;
  dmrg3s_status s;
  Scratch scr(c, st);
  DevSite& nbs = S.M[nb];
  SiteLayout nnl;
  if (dir == 1)
    make_site_from(nbs.lay.nsym, nbs.lay.d, nbs.lay.qp, nbnd, nbs.lay.right, &nnl);
  else
    make_site_from(nbs.lay.nsym, nbs.lay.d, nbs.lay.qp, nbs.lay.left, nbnd, &nnl);
  GemmStage g;
  for (const Block& ob : nnl.blocks) {
    const int ss = ob.a;
    std::vector<GemmSeg> sg;
    if (dir == 1) {       // B~[s](kn, j2) = SV_kn (nk x base) . B[s](jbase, j2)
      const int kn = ob.b;
      const Sector& sc = secs[sec_of_new[kn]];
      if (sc.base > 0) {
        const int bi = nbs.lay.block_of(ss, sc.jbase);
        if (bi >= 0 && nbs.lay.blocks[bi].c == ob.c) {
          GemmSeg q{};
          q.offA = rem_off[kn];
          q.lda = (int32_t)sc.base;
          q.offB = nbs.lay.blocks[bi].off;
          q.ldb = (int32_t)nbs.lay.blocks[bi].cols;
          q.K = (int32_t)sc.base;
          q.scale = 1.0;
          sg.push_back(q);
        }
      }
    } else {              // A~[s](i2, kn) = A[s](i2, jbase) . US_kn (base x nk)
      const int kn = ob.c;
      const Sector& sc = secs[sec_of_new[kn]];
      if (sc.base > 0) {
        const int bi = nbs.lay.block_of(ss, ob.b);
        if (bi >= 0 && nbs.lay.blocks[bi].c == sc.jbase) {
          GemmSeg q{};
          q.offA = nbs.lay.blocks[bi].off;
          q.lda = (int32_t)nbs.lay.blocks[bi].cols;
          q.offB = rem_off[kn];
          q.ldb = (int32_t)sc.keep;
          q.K = (int32_t)sc.base;
          q.scale = 1.0;
          sg.push_back(q);
        }
      }
    }
    g.add(ob.off, (int)ob.cols, (int)ob.rows, (int)ob.cols, sg);
  }
  double* nbdata;
  if ((s = scr.get(&nbdata, nnl.size))) return s;
  if (dir == 1) {
    if ((s = run_gemm(c, g, t.rem, t.rem_size, nbs.data, nbs.lay.size, nbdata, nnl.size, st))) return s;
  } else {
    if ((s = run_gemm(c, g, nbs.data, nbs.lay.size, t.rem, t.rem_size, nbdata, nnl.size, st))) return s;
  }
  dfree(t.rem, st);
  t.rem = nullptr;
  dfree(nbs.data, st);
  nbs.lay = nnl;
  nbs.data = scr.keep(nbdata);
  return DMRG3S_OK;
}

dmrg3s_status local_update(State& S, int dir, double alpha, const Opts& o, Info* info,
                           cudaStream_t st) {
  Context* c = S.c;
  const int i = S.centre;
  const int nb = i + dir;
  if (nb < 0 || nb >= S.n) return fail(c, DMRG3S_ERR_ARG, "local update would leave the chain");
  if (!S.Lenv[i].valid || !S.Renv[i].valid)
    return fail(c, DMRG3S_ERR_ARG, "environments of the centre site are not built");
  dmrg3s_status s;
  DevSite& m = S.M[i];
  const MpoLayout& w = S.W[i];
  Profiler& pr = c->prof;
  Scratch scr(c, st);   // every buffer of the update, freed on any exit
  auto phase = [&](int kind) { return pr.on ? pr.begin(kind, 0.0, 0.0, st) : -1; };
  auto done = [&](int id) {
    if (id >= 0) pr.end(id, st);
  };
  // ---- 1. eigensolver
  int ph = phase(kProfEig);
  if (o.optimise) {
    const DevicePlan* hp;
    if ((s = heff_plan(c, S.Lenv[i].lay, w, S.Renv[i].lay, m.lay, &hp))) return s;
    size_t cursor = (size_t)plan_ws_doubles(hp->host, o.prec) * sizeof(double);
    double lam = 0.0;
    int it = 0;
    if ((s = lanczos_run(c, *hp, S.Lenv[i].data, S.Renv[i].data, m.data, m.lay.size, o.kmax, lanczos_tol(o),
                         cursor, st, &lam, &it, o.prec)))
      return s;
    info->lambda = lam;
    info->iters = it;
  } else {
    if ((s = rayleigh(S, i, m.data, st, &info->lambda))) return s;
    info->iters = 0;
  }
  done(ph);
  // ---- 2. expansion term
  ph = phase(kProfExpand);
  const bool expand = alpha != 0.0;
  const Bond& old = dir == 1 ? m.lay.right : m.lay.left;
  FusedBond fp;      // P part only
  SiteLayout pl;
  double* P = nullptr;
  if (expand) {
    fuse_bond(old, dir == 1 ? w.wr : w.wl, dir == 1 ? w.tr : w.tl, false, &fp);
    if (dir == 1)
      make_site_from(m.lay.nsym, m.lay.d, m.lay.qp, m.lay.left, fp.bond, &pl);
    else
      make_site_from(m.lay.nsym, m.lay.d, m.lay.qp, fp.bond, m.lay.right, &pl);
    const DevicePlan* ep;
    const DevEnv& env = dir == 1 ? S.Lenv[i] : S.Renv[i];
    if ((s = expand_plan(c, dir, env.lay, w, m.lay, pl, fp, &ep))) return s;
    if ((size_t)ep->host.ws1 * sizeof(double) > c->ws_bytes)
      return fail(c, DMRG3S_ERR_OOM, "context workspace too small for the expansion");
    if ((s = scr.get(&P, pl.size))) return s;
    const double* g1A = dir == 1 ? env.data : m.data;
    const double* g1B = dir == 1 ? m.data : env.data;
    if ((s = run_plan(c, *ep, g1A, g1B, reinterpret_cast<double*>(c->ws), P, alpha, nullptr, nullptr,
                      nullptr, st)))
      return s;
  }
  done(ph);
  ph = phase(kProfSvd);
  // ---- 3. sectors of M~ = [M* P] (L->R) or [M*; P] (R->L), gathered
  Trunc t;
  prepare_truncation(m.lay, dir, expand, fp, pl, o.svd, o.prec, &t);
  double* X;
  if ((s = scr.get(&X, t.xoff))) return s;
  cudaMemsetAsync(X, 0, (size_t)std::max<int64_t>(t.xoff, 1) * sizeof(double), st);
  if ((s = run_copies(c, t.gather_m, m.data, m.lay.size, X, t.xoff, nullptr, 0, st))) return s;
  if (expand && (s = run_copies(c, t.gather_p, P, pl.size, X, t.xoff, nullptr, 0, st))) return s;
  scr.drop(P);
  // ---- 4. SVD per sector (FP64, on the tall orientation): cuSOLVER gesvd
  // runs the independent sectors concurrently on the workers' streams; the
  // Jacobi SVD (svd.cu) runs every sector in each of its launches.  The SVD
  // overwrites its input: the projected remainder reads a copy of X, which
  // also restores X when the Jacobi sweeps do not converge.
  double *F, *Sv, *dinfo_d, *X0 = nullptr;
  if ((s = scr.get(&F, t.foff)) || (s = scr.get(&Sv, t.soff)) ||
      (s = scr.get(&dinfo_d, (int64_t)t.secs.size() + 1)))
    return s;
  if (t.any_proj) {
    if ((s = scr.get(&X0, t.xoff))) return s;
    if ((s = cuda_ok(c, cudaMemcpyAsync(X0, X, (size_t)t.xoff * sizeof(double),
                                        cudaMemcpyDeviceToDevice, st), "copy of M~")))
      return s;
  }
  std::vector<double> hs;
  if ((s = svd_all(S, t.method, t.secs, X, X0, t.xoff, F, Sv, reinterpret_cast<int*>(dinfo_d), t.soff,
                   &hs, &info->svd_fallback, &info->svd_sweeps, st)))
    return s;
  scr.drop(X);
  scr.drop(dinfo_d);
  if ((s = truncate_centre(S, dir, o, t, F, Sv, X0, hs.data(), info, st))) return s;
  scr.drop(X0);
  scr.drop(F);
  scr.drop(Sv);
  done(ph);
  ph = phase(kProfRemainder);
  // ---- 5. remainder into the neighbour
  if ((s = update_neighbour(S, dir, nb, t, st))) return s;
  done(ph);
  ph = phase(kProfEnv);
  // ---- 6. environment of the truncated tensor; the neighbour's old one is stale
  if (dir == 1) {
    S.Renv[i].valid = false;
    if ((s = build_env(S, i, 1, st))) return s;
  } else {
    S.Lenv[i].valid = false;
    if ((s = build_env(S, i, -1, st))) return s;
  }
  S.centre = nb;
  done(ph);
  ph = phase(kProfEnergy);
  // ---- 7. energy after truncation at the neighbour
  if ((s = rayleigh(S, nb, S.M[nb].data, st, &info->e_f))) return s;
  done(ph);
  return cuda_ok(c, cudaGetLastError(), "local update");
}

// ---- batched local updates: one update on each of several states (the
// chains of a batch, one context), each contraction stage one launch over all
// of them.  The operands of the merged launches are copied into arenas (every
// tensor at a multiple of 32 elements) and the results copied back out.

inline int64_t align32(int64_t v) { return (v + 31) / 32 * 32; }

struct BItem {
  State* S = nullptr;
  int dir = 1;
  double alpha = 0.0;
  Opts o;
  Info info;
  bool expand = false;
  FusedBond fp;          // P part of the expanded bond
  SiteLayout pl;         // layout of P
  const double* P = nullptr;   // P inside the expansion arena
  Trunc t;
  int64_t xb = 0, fb = 0, sb = 0;   // bases of this update in the combined X, F, Sv
};

dmrg3s_status upload_merged(Context* c, Kind kind, const std::vector<PlanPart>& parts, int64_t nA1,
                            int64_t nB1, int64_t nOut2, int64_t nA3, int64_t nB3, int64_t nC3,
                            std::unique_ptr<DevicePlan>* out) {
  Plan mp;
  std::string err;
  dmrg3s_status s = merge_plans(kind, parts, nA1, nB1, nOut2, nA3, nB3, nC3, &mp, &err);
  if (s) return fail(c, s, "merged plan: " + err);
  if ((s = upload_plan(std::move(mp), out)))
    return fail(c, s, "uploading a merged contraction plan failed");
  return DMRG3S_OK;
}

dmrg3s_status copy_in(Context* c, double* dst, const double* src, int64_t n, cudaStream_t st) {
  if (n <= 0) return DMRG3S_OK;
  return cuda_ok(c, cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    st), "arena copy");
}

// Step 1 for every item: one Lanczos recursion per precision over all items
// of that precision (merged H_eff plans).
dmrg3s_status batch_eig(Context* c, std::vector<BItem>& items, cudaStream_t st) {
  dmrg3s_status s;
  const dmrg3s_precision precs[3] = {DMRG3S_FP64, DMRG3S_TF32X3, DMRG3S_TF32};
  for (dmrg3s_precision prec : precs) {
    std::vector<BItem*> g;
    for (BItem& it : items)
      if (it.o.optimise && it.o.prec == prec) g.push_back(&it);
    if (g.empty()) continue;
    if (g.size() == 1) {   // one problem: its own cached plan, no arenas
      BItem& it = *g[0];
      State& S = *it.S;
      const int i = S.centre;
      const DevicePlan* hp;
      if ((s = heff_plan(c, S.Lenv[i].lay, S.W[i], S.Renv[i].lay, S.M[i].lay, &hp))) return s;
      const size_t cursor = (size_t)plan_ws_doubles(hp->host, prec) * sizeof(double);
      if ((s = lanczos_run(c, *hp, S.Lenv[i].data, S.Renv[i].data, S.M[i].data, S.M[i].lay.size,
                           it.o.kmax, lanczos_tol(it.o), cursor, st, &it.info.lambda, &it.info.iters, prec)))
        return s;
      continue;
    }
    std::vector<PlanPart> parts(g.size());
    std::vector<LzSpec> specs(g.size());
    int64_t nL = 0, nR = 0, nX = 0;
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      const DevicePlan* hp;
      if ((s = heff_plan(c, S.Lenv[i].lay, S.W[i], S.Renv[i].lay, S.M[i].lay, &hp))) return s;
      PlanPart& q = parts[k];
      q.p = &hp->host;
      q.oA1 = nL;
      q.oB1 = nX;
      q.oB3 = nR;
      q.oC3 = nX;
      specs[k] = LzSpec{nX, S.M[i].lay.size, g[k]->o.kmax, lanczos_tol(g[k]->o)};
      nL += align32(S.Lenv[i].lay.size);
      nR += align32(S.Renv[i].lay.size);
      nX += align32(S.M[i].lay.size);
    }
    std::unique_ptr<DevicePlan> dp;
    if ((s = upload_merged(c, Kind::Heff, parts, nL, nX, 0, 0, nR, nX, &dp))) return s;
    Scratch scr(c, st);
    double *La, *Ra, *Xa;
    if ((s = scr.get(&La, nL)) || (s = scr.get(&Ra, nR)) || (s = scr.get(&Xa, nX))) return s;
    cudaMemsetAsync(Xa, 0, (size_t)nX * sizeof(double), st);
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      if ((s = copy_in(c, La + parts[k].oA1, S.Lenv[i].data, S.Lenv[i].lay.size, st)) ||
          (s = copy_in(c, Ra + parts[k].oB3, S.Renv[i].data, S.Renv[i].lay.size, st)) ||
          (s = copy_in(c, Xa + parts[k].oB1, S.M[i].data, S.M[i].lay.size, st)))
        return s;
    }
    const size_t cursor = (size_t)plan_ws_doubles(dp->host, prec) * sizeof(double);
    std::vector<double> theta;
    std::vector<int> iters;
    if ((s = lanczos_batch(c, *dp, La, Ra, Xa, nX, specs, cursor, st, prec, &theta, &iters)))
      return s;
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      if ((s = copy_in(c, S.M[i].data, Xa + parts[k].oB1, S.M[i].lay.size, st))) return s;
      g[k]->info.lambda = theta[k];
      g[k]->info.iters = iters[k];
    }
    // the merged tables are freed (cudaFree) only after the device is done with them
    if ((s = cuda_ok(c, cudaStreamSynchronize(st), "batched eigensolver"))) return s;
  }
  for (BItem& it : items)
    if (!it.o.optimise) {
      if ((s = rayleigh(*it.S, it.S->centre, it.S->M[it.S->centre].data, st, &it.info.lambda)))
        return s;
      it.info.iters = 0;
    }
  return DMRG3S_OK;
}

// Step 2 for every item with alpha != 0: one merged expansion launch set per
// direction (alpha folded into each item's MPO coefficients); every item's P
// stays in the arena `Pa` (owned by the caller's scratch) until gathered.
dmrg3s_status batch_expand(Context* c, std::vector<BItem>& items, Scratch& keep, cudaStream_t st) {
  dmrg3s_status s;
  for (BItem& it : items) {
    it.expand = it.alpha != 0.0;
    if (!it.expand) continue;
    State& S = *it.S;
    const int i = S.centre;
    const SiteLayout& ml = S.M[i].lay;
    const MpoLayout& w = S.W[i];
    const Bond& old = it.dir == 1 ? ml.right : ml.left;
    fuse_bond(old, it.dir == 1 ? w.wr : w.wl, it.dir == 1 ? w.tr : w.tl, false, &it.fp);
    if (it.dir == 1)
      make_site_from(ml.nsym, ml.d, ml.qp, ml.left, it.fp.bond, &it.pl);
    else
      make_site_from(ml.nsym, ml.d, ml.qp, it.fp.bond, ml.right, &it.pl);
  }
  for (int dir = -1; dir <= 1; dir += 2) {
    std::vector<BItem*> g;
    for (BItem& it : items)
      if (it.expand && it.dir == dir) g.push_back(&it);
    if (g.empty()) continue;
    std::vector<PlanPart> parts(g.size());
    int64_t nE = 0, nM = 0, nP = 0;
    std::vector<int64_t> oE(g.size()), oM(g.size()), oP(g.size());
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      const DevEnv& env = dir == 1 ? S.Lenv[i] : S.Renv[i];
      const DevicePlan* ep;
      if ((s = expand_plan(c, dir, env.lay, S.W[i], S.M[i].lay, g[k]->pl, g[k]->fp, &ep))) return s;
      oE[k] = nE;
      oM[k] = nM;
      oP[k] = nP;
      nE += align32(env.lay.size);
      nM += align32(S.M[i].lay.size);
      nP += align32(g[k]->pl.size);
      PlanPart& q = parts[k];
      q.p = &ep->host;
      q.oA1 = dir == 1 ? oE[k] : oM[k];
      q.oB1 = dir == 1 ? oM[k] : oE[k];
      q.oOut2 = oP[k];
      q.c2scale = g[k]->alpha;
    }
    std::unique_ptr<DevicePlan> dp;
    const Kind kind = dir == 1 ? Kind::ExpandLR : Kind::ExpandRL;
    if ((s = upload_merged(c, kind, parts, dir == 1 ? nE : nM, dir == 1 ? nM : nE, nP, 0, 0, 0, &dp)))
      return s;
    if ((size_t)dp->host.ws1 * sizeof(double) > c->ws_bytes)
      return fail(c, DMRG3S_ERR_OOM, "context workspace too small for the expansion");
    Scratch scr(c, st);
    double *Ea, *Ma, *Pa;
    if ((s = scr.get(&Ea, nE)) || (s = scr.get(&Ma, nM)) || (s = keep.get(&Pa, nP))) return s;
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      const DevEnv& env = dir == 1 ? S.Lenv[i] : S.Renv[i];
      if ((s = copy_in(c, Ea + oE[k], env.data, env.lay.size, st)) ||
          (s = copy_in(c, Ma + oM[k], S.M[i].data, S.M[i].lay.size, st)))
        return s;
      g[k]->P = Pa + oP[k];
    }
    if ((s = run_plan(c, *dp, dir == 1 ? Ea : Ma, dir == 1 ? Ma : Ea, reinterpret_cast<double*>(c->ws),
                      Pa, 1.0, nullptr, nullptr, nullptr, st)))
      return fail(c, s, "merged expansion launch");
    if ((s = cuda_ok(c, cudaStreamSynchronize(st), "batched expansion"))) return s;
  }
  return DMRG3S_OK;
}

// Steps 3 to 5 for every item: the sectors of every item gathered into one
// buffer, the SVD of all sectors of all items in one call (cuSOLVER lanes or
// the Jacobi launches over every sector), then per item the selection, the new
// centre tensor and the neighbour.
dmrg3s_status batch_truncate(Context* c, std::vector<BItem>& items, dmrg3s_svd_method method,
                             cudaStream_t st) {
  dmrg3s_status s;
  int64_t nX = 0, nF = 0, nS = 0;
  size_t nsec = 0;
  bool any_proj = false;
  dmrg3s_svd_method resolved = method == DMRG3S_SVD_AUTO ? DMRG3S_SVD_GESVD : method;
  for (BItem& it : items) {
    State& S = *it.S;
    prepare_truncation(S.M[S.centre].lay, it.dir, it.expand, it.fp, it.pl, method, it.o.prec,
                       &it.t);
    if (it.t.method == DMRG3S_SVD_JACOBI) resolved = DMRG3S_SVD_JACOBI;   // one call for all
    it.xb = nX;
    it.fb = nF;
    it.sb = nS;
    nX += align32(it.t.xoff);
    nF += align32(it.t.foff);
    nS += align32(it.t.soff);
    nsec += it.t.secs.size();
    any_proj = any_proj || it.t.any_proj;
  }
  method = resolved;
  any_proj = any_proj || method == DMRG3S_SVD_JACOBI;
  Scratch scr(c, st);
  double *X, *F, *Sv, *dinfo_d, *X0 = nullptr;
  if ((s = scr.get(&X, nX)) || (s = scr.get(&F, nF)) || (s = scr.get(&Sv, nS)) ||
      (s = scr.get(&dinfo_d, (int64_t)nsec + 1)))
    return s;
  cudaMemsetAsync(X, 0, (size_t)std::max<int64_t>(nX, 1) * sizeof(double), st);
  std::vector<Sector> all;
  all.reserve(nsec);
  for (BItem& it : items) {
    State& S = *it.S;
    const DevSite& m = S.M[S.centre];
    if ((s = run_copies(c, it.t.gather_m, m.data, m.lay.size, X + it.xb, it.t.xoff, nullptr, 0, st)))
      return s;
    if (it.expand &&
        (s = run_copies(c, it.t.gather_p, it.P, it.pl.size, X + it.xb, it.t.xoff, nullptr, 0, st)))
      return s;
    for (Sector sc : it.t.secs) {
      sc.off += it.xb;
      sc.offU += it.fb;
      sc.offVT += it.fb;
      sc.offS += it.sb;
      all.push_back(sc);
    }
  }
  if (any_proj) {
    if ((s = scr.get(&X0, nX))) return s;
    if ((s = cuda_ok(c, cudaMemcpyAsync(X0, X, (size_t)nX * sizeof(double), cudaMemcpyDeviceToDevice,
                                        st), "copy of M~")))
      return s;
  }
  std::vector<double> hs;
  bool fallback = false;
  int sweeps = 0;
  if ((s = svd_all(*items[0].S, method, all, X, X0, nX, F, Sv, reinterpret_cast<int*>(dinfo_d), nS,
                   &hs, &fallback, &sweeps, st)))
    return s;
  scr.drop(X);
  for (BItem& it : items) {
    it.info.svd_fallback = fallback;
    it.info.svd_sweeps = sweeps;
    State& S = *it.S;
    if ((s = truncate_centre(S, it.dir, it.o, it.t, F + it.fb, Sv + it.sb, X0 ? X0 + it.xb : nullptr,
                             hs.data() + it.sb, &it.info, st)) ||
        (s = update_neighbour(S, it.dir, S.centre + it.dir, it.t, st)))
      return s;
  }
  return DMRG3S_OK;
}

// Step 6 for every item: the environment of the truncated centre tensor, one
// merged launch set per direction; the centres then move to the neighbours.
dmrg3s_status batch_env(Context* c, std::vector<BItem>& items, cudaStream_t st) {
  dmrg3s_status s;
  for (int dir = -1; dir <= 1; dir += 2) {
    std::vector<BItem*> g;
    for (BItem& it : items)
      if (it.dir == dir) g.push_back(&it);
    if (g.empty()) continue;
    std::vector<PlanPart> parts(g.size());
    std::vector<EnvLayout> outl(g.size());
    std::vector<int64_t> oE(g.size()), oA(g.size()), oO(g.size());
    int64_t nE = 0, nA = 0, nO = 0;
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      const MpoLayout& w = S.W[i];
      const DevSite& a = S.M[i];
      const DevEnv& src = dir == 1 ? S.Lenv[i] : S.Renv[i];
      if (!src.valid)
        return fail(c, DMRG3S_ERR_ARG, "environment recursion from an invalid environment");
      make_env_from(a.lay.nsym, dir == 1 ? w.wr : w.wl, dir == 1 ? w.tr : w.tl,
                    dir == 1 ? a.lay.right : a.lay.left, &outl[k]);
      const DevicePlan* p;
      if ((s = env_plan(c, dir, src.lay, w, a.lay, outl[k], &p))) return s;
      oE[k] = nE;
      oA[k] = nA;
      oO[k] = nO;
      nE += align32(src.lay.size);
      nA += align32(a.lay.size);
      nO += align32(outl[k].size);
      PlanPart& q = parts[k];
      q.p = &p->host;
      q.oA1 = dir == 1 ? oE[k] : oA[k];
      q.oB1 = dir == 1 ? oA[k] : oE[k];
      q.oA3 = oA[k];
      q.oC3 = oO[k];
    }
    std::unique_ptr<DevicePlan> dp;
    const Kind kind = dir == 1 ? Kind::EnvLR : Kind::EnvRL;
    if ((s = upload_merged(c, kind, parts, dir == 1 ? nE : nA, dir == 1 ? nA : nE, 0, nA, 0, nO,
                           &dp)))
      return s;
    if ((size_t)(dp->host.ws1 + dp->host.ws2) * sizeof(double) > c->ws_bytes)
      return fail(c, DMRG3S_ERR_OOM, "context workspace too small for the environment update");
    Scratch scr(c, st);
    double *Ea, *Aa, *Oa;
    if ((s = scr.get(&Ea, nE)) || (s = scr.get(&Aa, nA)) || (s = scr.get(&Oa, nO))) return s;
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      const DevEnv& src = dir == 1 ? S.Lenv[i] : S.Renv[i];
      if ((s = copy_in(c, Ea + oE[k], src.data, src.lay.size, st)) ||
          (s = copy_in(c, Aa + oA[k], S.M[i].data, S.M[i].lay.size, st)))
        return s;
    }
    double* ws1 = reinterpret_cast<double*>(c->ws);
    double* ws2 = ws1 + dp->host.ws1;
    if ((s = run_plan(c, *dp, dir == 1 ? Ea : Aa, dir == 1 ? Aa : Ea, ws1, ws2, 1.0, Aa, ws2, Oa,
                      st)))
      return fail(c, s, "merged environment update launch");
    for (size_t k = 0; k < g.size(); ++k) {
      State& S = *g[k]->S;
      const int i = S.centre;
      double* nd;
      if ((s = dalloc(c, &nd, outl[k].size, st))) return s;
      if ((s = copy_in(c, nd, Oa + oO[k], outl[k].size, st))) {
        dfree(nd, st);
        return s;
      }
      // the environment built from the truncated tensor; the one on its other
      // side (built from the old tensor) is stale
      DevEnv& dst = dir == 1 ? S.Lenv[i + 1] : S.Renv[i - 1];
      (dir == 1 ? S.Renv[i] : S.Lenv[i]).valid = false;
      dfree(dst.data, st);
      dst.data = nd;
      dst.lay = outl[k];
      dst.valid = true;
      S.centre = i + dir;
    }
    if ((s = cuda_ok(c, cudaStreamSynchronize(st), "batched environment update"))) return s;
  }
  return DMRG3S_OK;
}

// Step 7 for every item: E_f = <x|H_eff|x> / <x|x> at the new centre, one
// merged FP64 H_eff launch set and one pair of reductions for all items.
dmrg3s_status batch_energy(Context* c, std::vector<BItem>& items, cudaStream_t st) {
  dmrg3s_status s;
  std::vector<PlanPart> parts(items.size());
  std::vector<std::pair<int64_t, int64_t>> ranges(items.size());
  int64_t nL = 0, nR = 0, nX = 0;
  for (size_t k = 0; k < items.size(); ++k) {
    State& S = *items[k].S;
    const int i = S.centre;
    if (!S.Lenv[i].valid || !S.Renv[i].valid)
      return fail(c, DMRG3S_ERR_ARG, "environments of the new centre are not built");
    const DevicePlan* hp;
    if ((s = heff_plan(c, S.Lenv[i].lay, S.W[i], S.Renv[i].lay, S.M[i].lay, &hp))) return s;
    PlanPart& q = parts[k];
    q.p = &hp->host;
    q.oA1 = nL;
    q.oB1 = nX;
    q.oB3 = nR;
    q.oC3 = nX;
    ranges[k] = {nX, S.M[i].lay.size};
    nL += align32(S.Lenv[i].lay.size);
    nR += align32(S.Renv[i].lay.size);
    nX += align32(S.M[i].lay.size);
  }
  std::unique_ptr<DevicePlan> dp;
  if ((s = upload_merged(c, Kind::Heff, parts, nL, nX, 0, 0, nR, nX, &dp))) return s;
  if ((size_t)(dp->host.ws1 + dp->host.ws2) * sizeof(double) > c->ws_bytes)
    return fail(c, DMRG3S_ERR_OOM, "context workspace too small for H_eff");
  std::vector<LzChunk> hch;
  std::vector<LzChain> hcn;
  lz_layout(ranges, 2 * plan_ctas(), &hch, &hcn);
  const int nch = (int)hch.size();
  Scratch scr(c, st);
  double *La, *Ra, *Xa, *Ya, *part, *tabs;
  const int64_t tab_doubles =
      (int64_t)((hch.size() * sizeof(LzChunk) + hcn.size() * sizeof(LzChain)) / sizeof(double)) + 2;
  if ((s = scr.get(&La, nL)) || (s = scr.get(&Ra, nR)) || (s = scr.get(&Xa, nX)) ||
      (s = scr.get(&Ya, nX)) || (s = scr.get(&part, 2 * (int64_t)nch)) ||
      (s = scr.get(&tabs, tab_doubles)))
    return s;
  LzChunk* dch = reinterpret_cast<LzChunk*>(tabs);
  LzChain* dcn = reinterpret_cast<LzChain*>(dch + nch);
  if ((s = cuda_ok(c, cudaMemcpyAsync(dch, hch.data(), sizeof(LzChunk) * nch,
                                      cudaMemcpyHostToDevice, st), "reduction tables")) ||
      (s = cuda_ok(c, cudaMemcpyAsync(dcn, hcn.data(), sizeof(LzChain) * hcn.size(),
                                      cudaMemcpyHostToDevice, st), "reduction tables")))
    return s;
  cudaMemsetAsync(Xa, 0, (size_t)nX * sizeof(double), st);
  for (size_t k = 0; k < items.size(); ++k) {
    State& S = *items[k].S;
    const int i = S.centre;
    if ((s = copy_in(c, La + parts[k].oA1, S.Lenv[i].data, S.Lenv[i].lay.size, st)) ||
        (s = copy_in(c, Ra + parts[k].oB3, S.Renv[i].data, S.Renv[i].lay.size, st)) ||
        (s = copy_in(c, Xa + parts[k].oB1, S.M[i].data, S.M[i].lay.size, st)))
      return s;
  }
  double* ws1 = reinterpret_cast<double*>(c->ws);
  double* ws2 = ws1 + dp->host.ws1;
  if ((s = run_plan(c, *dp, La, Xa, ws1, ws2, 1.0, ws2, Ra, Ya, st)))
    return fail(c, s, "merged H_eff launch");
  launch_lz_dots(Xa, nX, 1, Ya, dch, nch, part, 1, st);                          // <x, Hx>
  launch_lz_update(nullptr, nX, 0, Xa, dch, nch, dcn, nullptr, 1, nullptr, part + nch, st);   // <x, x>
  if ((s = pinned_reserve(c, 2 * (size_t)nch))) return s;
  double* pin = c->pinned_big;
  if ((s = cuda_ok(c, cudaMemcpyAsync(pin, part, sizeof(double) * 2 * nch, cudaMemcpyDeviceToHost,
                                      st), "energy read-back")) ||
      (s = cuda_ok(c, cudaStreamSynchronize(st), "batched energy")))
    return s;
  for (size_t k = 0; k < items.size(); ++k) {
    double num = 0.0, den = 0.0;
    for (int b = 0; b < hcn[k].nc; ++b) {
      num += pin[hcn[k].c0 + b];
      den += pin[nch + hcn[k].c0 + b];
    }
    items[k].info.e_f = den > 0.0 ? num / den : 0.0;
  }
  return DMRG3S_OK;
}

// One local update on every item's state (each in its own direction, with its
// own alpha and options); the same steps as local_update, batched.
dmrg3s_status local_update_batch(Context* c, std::vector<BItem>& items, dmrg3s_svd_method method,
                                 cudaStream_t st) {
  dmrg3s_status s;
  for (BItem& it : items) {
    State& S = *it.S;
    const int i = S.centre, nb = i + it.dir;
    if (nb < 0 || nb >= S.n) return fail(c, DMRG3S_ERR_ARG, "local update would leave the chain");
    if (!S.Lenv[i].valid || !S.Renv[i].valid)
      return fail(c, DMRG3S_ERR_ARG, "environments of the centre site are not built");
    it.info = Info();
  }
  Profiler& pr = c->prof;
  auto phase = [&](int kind) { return pr.on ? pr.begin(kind, 0.0, 0.0, st) : -1; };
  auto done = [&](int id) {
    if (id >= 0) pr.end(id, st);
  };
  int ph = phase(kProfEig);
  if ((s = batch_eig(c, items, st))) return s;
  done(ph);
  ph = phase(kProfExpand);
  Scratch keep(c, st);    // the expansion terms, until gathered
  if ((s = batch_expand(c, items, keep, st))) return s;
  done(ph);
  ph = phase(kProfSvd);
  if ((s = batch_truncate(c, items, method, st))) return s;
  done(ph);
  ph = phase(kProfEnv);
  if ((s = batch_env(c, items, st))) return s;
  done(ph);
  ph = phase(kProfEnergy);
  if ((s = batch_energy(c, items, st))) return s;
  done(ph);
  return cuda_ok(c, cudaGetLastError(), "batched local update");
}

dmrg3s_status boundary_env(State& S, const dmrg3s_env* user, bool left, cudaStream_t st) {
  Context* c = S.c;
  const int i = left ? 0 : S.n - 1;
  DevEnv& e = left ? S.Lenv[0] : S.Renv[S.n - 1];
  const SiteLayout& a = S.M[i].lay;
  const MpoLayout& w = S.W[i];
  std::string err;
  dmrg3s_status s;
  if (user) {
    EnvLayout el;
    if ((s = make_env(user, &el, &err))) return fail(c, s, err);
    if ((s = check_env(el, left ? a.left : a.right, left ? w.wl : w.wr, left ? w.tl : w.tr,
                       left ? "left boundary" : "right boundary", &err)))
      return fail(c, s, err);
    if (!user->data) return fail(c, DMRG3S_ERR_ARG, "boundary environment without data");
    if ((s = dalloc(c, &e.data, el.size, st))) return s;
    cudaMemcpyAsync(e.data, user->data, (size_t)el.size * sizeof(double), cudaMemcpyDeviceToDevice, st);
    e.lay = el;
  } else {
    const Bond& b = left ? a.left : a.right;
    if ((left ? w.wl : w.wr) != 1 || b.total != 1)
      return fail(c, DMRG3S_ERR_SHAPE, "a trivial boundary needs a bond and an MPO bond of dimension 1");
    EnvLayout el;
    make_env_from(a.nsym, 1, left ? w.tl : w.tr, b, &el);
    if (el.size != 1) return fail(c, DMRG3S_ERR_QN, "trivial boundary charges do not match");
    if ((s = dalloc(c, &e.data, 1, st))) return s;
    static const double one = 1.0;
    cudaMemcpyAsync(e.data, &one, sizeof(double), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    e.lay = el;
  }
  e.valid = true;
  return DMRG3S_OK;
}

// Frees everything a (possibly partly built) state holds, after the device
// has finished the work that uses it.
void release_state(State* S) {
  use_device(S->c);
  cudaDeviceSynchronize();
  for (auto& m : S->M) cudaFree(m.data);
  for (auto& e : S->Lenv) cudaFree(e.data);
  for (auto& e : S->Renv) cudaFree(e.data);
  for (SvdWorker& w : S->svd) lane_destroy(&w);
  if (S->svd_in) cudaEventDestroy(S->svd_in);
  delete S;
}

struct StateGuard {       // releases a state under construction on an error exit
  State* S;
  ~StateGuard() {
    if (S) release_state(S);
  }
};

}  // namespace
}  // namespace dmrg3s

using namespace dmrg3s;

extern "C" {

dmrg3s_status dmrg3s_state_create(dmrg3s_ctx ctx, int32_t nsites, const dmrg3s_mpo_site* W,
                                  const dmrg3s_site* M, const dmrg3s_env* left_env,
                                  const dmrg3s_env* right_env, int32_t centre,
                                  dmrg3s_state* out, dmrg3s_stream stream) {
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c || !W || !M || !out || nsites < 1) return fail(c, DMRG3S_ERR_ARG, "bad argument");
  if (centre < 0 || centre >= nsites) return fail(c, DMRG3S_ERR_ARG, "centre out of range");
  *out = nullptr;
  dmrg3s_status s;
  if ((s = use_device(c))) return s;
  State* S = new (std::nothrow) State();
  if (!S) return fail(c, DMRG3S_ERR_OOM, "state");
  StateGuard guard{S};
  S->c = c;
  S->n = nsites;
  S->W.resize(nsites);
  S->M.resize(nsites);
  S->Lenv.resize(nsites);
  S->Renv.resize(nsites);
  std::string err;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < nsites; ++i) {
    if ((s = make_mpo(&W[i], &S->W[i], &err)) || (s = make_site(&M[i], &S->M[i].lay, &err)) ||
        (s = check_site_mpo(S->M[i].lay, S->W[i], &err)))
      return fail(c, s, "site " + std::to_string(i) + ": " + err);
    if (i > 0) {
      if (!same_bond(S->M[i - 1].lay.right, S->M[i].lay.left))
        return fail(c, DMRG3S_ERR_SHAPE, "bond " + std::to_string(i) + " differs between sites");
      if (S->W[i - 1].wr != S->W[i].wl || !same_charges(S->W[i - 1].tr, S->W[i].tl))
        return fail(c, DMRG3S_ERR_SHAPE, "MPO bond " + std::to_string(i) + " differs between sites");
    }
    if (!M[i].data) return fail(c, DMRG3S_ERR_ARG, "site without data");
    if ((s = dalloc(c, &S->M[i].data, S->M[i].lay.size, st))) return s;
    cudaMemcpyAsync(S->M[i].data, M[i].data, (size_t)S->M[i].lay.size * sizeof(double),
                    cudaMemcpyDeviceToDevice, st);
  }
  S->svd.resize(svd_lanes());
  for (SvdWorker& w : S->svd)
    if ((s = lane_create(c, &w))) return s;
  if (cudaEventCreateWithFlags(&S->svd_in, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, DMRG3S_ERR_CUDA, "SVD event");
  if ((s = boundary_env(*S, left_env, true, st)) || (s = boundary_env(*S, right_env, false, st)))
    return s;
  for (int i = 0; i < centre; ++i)
    if ((s = build_env(*S, i, 1, st))) return s;
  for (int i = nsites - 1; i > centre; --i)
    if ((s = build_env(*S, i, -1, st))) return s;
  S->centre = centre;
  if ((s = rayleigh(*S, centre, S->M[centre].data, st, &S->e_in))) return s;
  guard.S = nullptr;
  *out = reinterpret_cast<dmrg3s_state>(S);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_state_destroy(dmrg3s_state state) {
  State* S = reinterpret_cast<State*>(state);
  if (!S) return DMRG3S_ERR_ARG;
  release_state(S);
  return DMRG3S_OK;
}

}  // extern "C"

namespace {
dmrg3s_status make_opts(Context* c, int32_t dir, const dmrg3s_update_opts* opts, Opts* o) {
  if (dir != 1 && dir != -1) return fail(c, DMRG3S_ERR_ARG, "dir must be +1 or -1");
  if (opts->precision != DMRG3S_FP64 && opts->precision != DMRG3S_TF32X3 &&
      opts->precision != DMRG3S_TF32)
    return fail(c, DMRG3S_ERR_ARG, "local update precision");
  if (opts->m_max < 1) return fail(c, DMRG3S_ERR_ARG, "m_max must be >= 1");
  if (opts->svd != DMRG3S_SVD_JACOBI && opts->svd != DMRG3S_SVD_GESVD &&
      opts->svd != DMRG3S_SVD_AUTO)
    return fail(c, DMRG3S_ERR_ARG, "SVD method");
  o->m_max = opts->m_max;
  o->kmax = opts->lanczos_kmax > 0 ? opts->lanczos_kmax : 40;
  o->tol = opts->lanczos_tol > 0 ? opts->lanczos_tol : 1e-10;
  o->eps = opts->trunc_eps > 0 ? opts->trunc_eps : 1e-12;
  o->optimise = opts->skip_eigensolver == 0;
  o->prec = opts->precision;
  o->svd = opts->svd;
  return DMRG3S_OK;
}

void report_info(State* S, const Info& inf, dmrg3s_update_info* info) {
  info->lambda = inf.lambda;
  info->energy_after = inf.e_f;
  info->energy_before = S->e_in;
  info->discarded_weight = inf.discarded;
  info->lanczos_iters = inf.iters;
  info->new_bond_dim = inf.new_dim;
  info->svd_fallback = inf.svd_fallback ? 1 : 0;
  info->svd_sweeps = inf.svd_sweeps;
  S->e_in = inf.e_f;
}

// Checks of a batch: distinct states of one context, one SVD method.
dmrg3s_status check_batch(const dmrg3s_state* states, int32_t n, Context** cout) {
  if (!states || n < 1) return DMRG3S_ERR_ARG;
  State* S0 = reinterpret_cast<State*>(states[0]);
  if (!S0) return DMRG3S_ERR_ARG;
  Context* c = S0->c;
  for (int k = 0; k < n; ++k) {
    State* S = reinterpret_cast<State*>(states[k]);
    if (!S) return fail(c, DMRG3S_ERR_ARG, "NULL state in a batch");
    if (S->c != c) return fail(c, DMRG3S_ERR_ARG, "the states of a batch share one context");
    for (int j = 0; j < k; ++j)
      if (states[j] == states[k]) return fail(c, DMRG3S_ERR_ARG, "a state appears twice in a batch");
  }
  *cout = c;
  return DMRG3S_OK;
}
}  // namespace

extern "C" {

dmrg3s_status dmrg3s_local_update(dmrg3s_state state, int32_t dir, double alpha,
                                  const dmrg3s_update_opts* opts, dmrg3s_update_info* info,
                                  dmrg3s_stream stream) {
  State* S = reinterpret_cast<State*>(state);
  if (!S || !opts || !info) return DMRG3S_ERR_ARG;
  Context* c = S->c;
  dmrg3s_status s;
  Opts o;
  if ((s = make_opts(c, dir, opts, &o))) return s;
  if ((s = use_device(c))) return s;
  Info inf;
  s = local_update(*S, dir, alpha, o, &inf, reinterpret_cast<cudaStream_t>(stream));
  if (s != DMRG3S_OK) return s;
  report_info(S, inf, info);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_local_update_batch(const dmrg3s_state* states, int32_t nstates,
                                        const int32_t* dirs, const double* alphas,
                                        const dmrg3s_update_opts* opts, dmrg3s_update_info* infos,
                                        dmrg3s_stream stream) {
  Context* c = nullptr;
  dmrg3s_status s;
  if ((s = check_batch(states, nstates, &c))) return s;
  if (!dirs || !alphas || !opts || !infos) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  std::vector<BItem> items(nstates);
  for (int k = 0; k < nstates; ++k) {
    if ((s = make_opts(c, dirs[k], &opts[k], &items[k].o))) return s;
    if (opts[k].svd != opts[0].svd)
      return fail(c, DMRG3S_ERR_ARG, "the updates of a batch use one SVD method");
    items[k].S = reinterpret_cast<State*>(states[k]);
    items[k].dir = dirs[k];
    items[k].alpha = alphas[k];
  }
  if ((s = use_device(c))) return s;
  if ((s = local_update_batch(c, items, opts[0].svd, reinterpret_cast<cudaStream_t>(stream))))
    return s;
  for (int k = 0; k < nstates; ++k) report_info(items[k].S, items[k].info, &infos[k]);
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_state_centre(dmrg3s_state state, int32_t* centre, double* energy) {
  State* S = reinterpret_cast<State*>(state);
  if (!S) return DMRG3S_ERR_ARG;
  if (centre) *centre = S->centre;
  if (energy) *energy = S->e_in;
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_state_site_info(dmrg3s_state state, int32_t i, int32_t* nsec_left,
                                     int32_t* q_left, int64_t* dim_left, int32_t* nsec_right,
                                     int32_t* q_right, int64_t* dim_right, int64_t* nelem) {
  State* S = reinterpret_cast<State*>(state);
  if (!S || i < 0 || i >= S->n) return DMRG3S_ERR_ARG;
  const SiteLayout& l = S->M[i].lay;
  auto put = [&](const Bond& b, int32_t* ns, int32_t* q, int64_t* dim) {
    if (ns) *ns = b.nsec();
    if (q && b.nsym)
      for (int k = 0; k < b.nsec(); ++k)
        for (int j = 0; j < b.nsym; ++j) q[(size_t)k * b.nsym + j] = b.q[k][j];
    if (dim)
      for (int k = 0; k < b.nsec(); ++k) dim[k] = b.dim[k];
  };
  put(l.left, nsec_left, q_left, dim_left);
  put(l.right, nsec_right, q_right, dim_right);
  if (nelem) *nelem = l.size;
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_state_site_copy(dmrg3s_state state, int32_t i, double* dst,
                                     dmrg3s_stream stream) {
  State* S = reinterpret_cast<State*>(state);
  if (!S || i < 0 || i >= S->n || !dst) return DMRG3S_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(dst, S->M[i].data, (size_t)S->M[i].lay.size * sizeof(double),
                                  cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DMRG3S_OK : fail(S->c, DMRG3S_ERR_CUDA, "site copy");
}

}  // extern "C"

namespace {

// Every G_i of the state (host, concatenated in site order; goff[i] = offset
// of site i) and <Psi|Psi>.
dmrg3s_status grad_all(State* S, cudaStream_t st, std::vector<double>* hGout,
                       std::vector<int64_t>* goffout, double* norm2) {
  Context* c = S->c;
  int64_t total = 0;
  std::vector<int64_t>& goff = *goffout;
  goff.assign(S->n, 0);
  for (int i = 0; i < S->n; ++i) {
    goff[i] = total;
    total += (int64_t)S->W[i].d * S->W[i].d * S->W[i].wl * S->W[i].wr;
  }
  dmrg3s_status s;
  if ((s = use_device(c))) return s;
  const int cen = S->centre;
  if (!S->Lenv[cen].valid || !S->Renv[cen].valid)
    return fail(c, DMRG3S_ERR_ARG, "environments of the centre are not valid");
  double* dG;
  if ((s = dalloc(c, &dG, total, st))) return s;
  // G_i for the centre and, walking outwards, for every other site with the
  // environment of the current tensors on the far side of the centre
  auto grad_at = [&](int i, const EnvLayout& ll, const double* L, const EnvLayout& rl,
                     const double* R) -> dmrg3s_status {
    GradPlan p;
    std::string err;
    dmrg3s_status r = plan_mpo_grad(ll, S->W[i], rl, S->M[i].lay, &p, &err);
    if (r) return fail(c, r, "site " + std::to_string(i) + ": " + err);
    return run_mpo_grad(c, p, L, S->M[i].data, R, dG + goff[i], st);
  };
  s = grad_at(cen, S->Lenv[cen].lay, S->Lenv[cen].data, S->Renv[cen].lay, S->Renv[cen].data);
  for (int dir = -1; dir <= 1 && !s; dir += 2) {
    // dir = -1: sites left of the centre (left environments stored, right
    // ones rebuilt); dir = +1: the mirror image
    EnvLayout lay = dir == -1 ? S->Renv[cen].lay : S->Lenv[cen].lay;
    const double* cur = dir == -1 ? S->Renv[cen].data : S->Lenv[cen].data;
    double* owned = nullptr;
    for (int i = cen + dir; i >= 0 && i < S->n && !s; i += dir) {
      EnvLayout nl;
      double* nd = nullptr;
      if ((s = env_step(*S, i - dir, dir, lay, cur, &nl, &nd, st))) break;
      dfree(owned, st);
      owned = nd;
      cur = nd;
      lay = nl;
      if (dir == -1) {
        if (!S->Lenv[i].valid) s = fail(c, DMRG3S_ERR_ARG, "left environment not valid");
        else s = grad_at(i, S->Lenv[i].lay, S->Lenv[i].data, lay, cur);
      } else {
        if (!S->Renv[i].valid) s = fail(c, DMRG3S_ERR_ARG, "right environment not valid");
        else s = grad_at(i, lay, cur, S->Renv[i].lay, S->Renv[i].data);
      }
    }
    dfree(owned, st);
  }
  double nrm = 0.0;
  if (!s) s = dot_host(c, S->M[cen].data, S->M[cen].data, S->M[cen].lay.size, st, &nrm);
  std::vector<double>& hG = *hGout;
  hG.assign(total, 0.0);
  if (!s && total > 0)
    s = cuda_ok(c, cudaMemcpyAsync(hG.data(), dG, (size_t)total * sizeof(double),
                                   cudaMemcpyDeviceToHost, st), "gradient read-back");
  dfree(dG, st);
  if (!s) s = cuda_ok(c, cudaStreamSynchronize(st), "gradient");
  if (s) return s;
  if (!(nrm > 0.0)) return fail(c, DMRG3S_ERR_NUMERIC, "zero norm of the centre tensor");
  *norm2 = nrm;
  return DMRG3S_OK;
}

}  // namespace

extern "C" {

dmrg3s_status dmrg3s_mpo_grad(dmrg3s_state state, double* G, const double* dW, int64_t len,
                              double* dE, double* norm2, dmrg3s_stream stream) {
  State* S = reinterpret_cast<State*>(state);
  if (!S) return DMRG3S_ERR_ARG;
  Context* c = S->c;
  int64_t total = 0;
  for (int i = 0; i < S->n; ++i) total += (int64_t)S->W[i].d * S->W[i].d * S->W[i].wl * S->W[i].wr;
  if ((G || dW) && len != total)
    return fail(c, DMRG3S_ERR_SHAPE, "len must be the summed d*d*wl*wr over the sites");
  std::vector<double> hG;
  std::vector<int64_t> goff;
  double nrm = 0.0;
  dmrg3s_status s = grad_all(S, reinterpret_cast<cudaStream_t>(stream), &hG, &goff, &nrm);
  if (s) return s;
  if (G && total > 0) std::memcpy(G, hG.data(), (size_t)total * sizeof(double));
  if (norm2) *norm2 = nrm;
  if (dE) {
    double acc = 0.0;
    if (dW)
      for (int64_t k = 0; k < total; ++k) acc += hG[k] * dW[k];
    *dE = acc / nrm;
  }
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_energy_grad(dmrg3s_state state, int32_t model, int32_t nparams,
                                 const double* params, double* energy, double* dE,
                                 dmrg3s_stream stream) {
  State* S = reinterpret_cast<State*>(state);
  if (!S) return DMRG3S_ERR_ARG;
  Context* c = S->c;
  if (!params || nparams != 2) return fail(c, DMRG3S_ERR_ARG, "nparams must be 2 with params");
  if (model != DMRG3S_MODEL_XXZ && model != DMRG3S_MODEL_HUBBARD)
    return fail(c, DMRG3S_ERR_UNSUPPORTED, "energy gradient: XXZ and HUBBARD only");
  // the model's MPO at params and at params + e_k (host builders)
  std::vector<dmrg3s_mpo> mp(nparams + 1, nullptr);
  struct Free {
    std::vector<dmrg3s_mpo>& v;
    ~Free() {
      for (dmrg3s_mpo m : v)
        if (m) dmrg3s_mpo_destroy(m);
    }
  } free_mpos{mp};
  for (int k = 0; k <= nparams; ++k) {
    double p[2] = {params[0], params[1]};
    if (k > 0) p[k - 1] += 1.0;
    dmrg3s_status s = dmrg3s_mpo_create(model, S->n, p, 0, nullptr, nullptr, &mp[k]);
    if (s) return fail(c, s, "energy gradient: model MPO");
  }
  // the state's MPO must be the model at params (same structure and entries)
  for (int i = 0; i < S->n; ++i) {
    dmrg3s_mpo_site w{};
    dmrg3s_mpo_get_site(mp[0], i, &w);
    const MpoLayout& sw = S->W[i];
    if (w.d != sw.d || w.wl != sw.wl || w.wr != sw.wr ||
        std::memcmp(w.W, sw.W.data(), sizeof(double) * sw.W.size()) != 0)
      return fail(c, DMRG3S_ERR_SHAPE,
                  "energy gradient: the state's MPO at site " + std::to_string(i) +
                      " is not the model at params");
  }
  std::vector<double> hG;
  std::vector<int64_t> goff;
  double nrm = 0.0;
  dmrg3s_status s = grad_all(S, reinterpret_cast<cudaStream_t>(stream), &hG, &goff, &nrm);
  if (s) return s;
  if (energy) {
    const int cen = S->centre;
    const std::vector<double>& Wc = S->W[cen].W;
    double acc = 0.0;
    for (size_t e = 0; e < Wc.size(); ++e) acc += hG[goff[cen] + e] * Wc[e];
    *energy = acc / nrm;
  }
  if (dE)
    for (int k = 0; k < nparams; ++k) {
      double acc = 0.0;
      for (int i = 0; i < S->n; ++i) {
        dmrg3s_mpo_site wk{}, w0{};
        dmrg3s_mpo_get_site(mp[k + 1], i, &wk);
        dmrg3s_mpo_get_site(mp[0], i, &w0);
        const int64_t ne = (int64_t)w0.d * w0.d * w0.wl * w0.wr;
        for (int64_t e = 0; e < ne; ++e) acc += hG[goff[i] + e] * (wk.W[e] - w0.W[e]);
      }
      dE[k] = acc / nrm;
    }
  return DMRG3S_OK;
}

}  // extern "C"

namespace {
// Adaptive mixing factor of Sec. VI with the thresholds documented in
// include/dmrg3s.h (dmrg3s_alpha_rule).
double alpha_update(const dmrg3s_alpha_rule& r, double alpha, double e_in, double lam, double e_f) {
  if (r.fixed) return alpha;
  const double d_o = lam - e_in, d_t = e_f - lam;
  if (std::fabs(d_o) < 1e-13 * std::max(std::fabs(lam), 1e-300))
    alpha *= r.down;
  else if (d_t < 0.0 || d_t / std::fabs(d_o) < r.target)
    alpha *= r.up;
  else if (d_t / std::fabs(d_o) > 1.0)
    alpha *= r.down * r.down;
  else
    alpha *= r.down;
  return std::min(std::max(alpha, r.alpha_min), r.alpha_max);
}
}  // namespace

namespace {
// The sweep schedule of one state: right-to-left then left-to-right passes
// of local updates with the adaptive alpha (Sec. VI), the precision ladder
// (dmrg3s_sweep_opts.switch_tol) and the convergence rule, advanced one
// local update at a time so that several states can share each step.
struct Sweeper {
  State* S = nullptr;
  const dmrg3s_alpha_rule* rule = nullptr;
  const dmrg3s_sweep_opts* opts = nullptr;
  double* energies = nullptr;
  dmrg3s_sweep_report* report = nullptr;
  dmrg3s_update_opts uo{};
  double alpha = 0.0, prev = 0.0, e = 0.0;
  bool final_stage = true, done = false;
  int final_sweeps = 0, sw = 0, pass = 0, k = 0;
  int64_t nupd = 0;
  std::chrono::steady_clock::time_point t0;

  dmrg3s_status init(Context* c) {
    if (S->n < 2) return fail(c, DMRG3S_ERR_ARG, "a sweep needs at least two sites");
    if (S->centre != S->n - 1)
      return fail(c, DMRG3S_ERR_ARG, "a sweep starts with the centre on the last site");
    if (opts->max_sweeps < 1) return fail(c, DMRG3S_ERR_ARG, "max_sweeps must be >= 1");
    const bool ladder = opts->switch_tol > 0.0;
    if (ladder && opts->final_precision != DMRG3S_FP64 &&
        opts->final_precision != DMRG3S_TF32X3 && opts->final_precision != DMRG3S_TF32)
      return fail(c, DMRG3S_ERR_ARG, "final precision");
    t0 = std::chrono::steady_clock::now();
    alpha = rule->alpha0;
    report->sweeps = 0;
    report->converged = 0;
    report->lanczos_iters = 0;
    report->svd_fallbacks = 0;
    report->bulk_sweeps = 0;
    report->pad = 0;
    uo = opts->update;
    final_stage = !ladder;       // without a ladder every sweep counts
    return DMRG3S_OK;
  }
  int dir() const { return pass == 0 ? -1 : 1; }
  // bookkeeping after the local update `inf` of this state
  void after(const dmrg3s_update_info& inf) {
    alpha = alpha_update(*rule, alpha, inf.energy_before, inf.lambda, inf.energy_after);
    if (opts->alphas) opts->alphas[nupd] = alpha;
    ++nupd;
    report->lanczos_iters += inf.lanczos_iters;
    report->svd_fallbacks += inf.svd_fallback;
    e = inf.energy_after;
    if (++k < S->n - 1) return;
    k = 0;
    if (++pass < 2) return;
    pass = 0;
    // end of a sweep
    if (energies) energies[sw] = e;
    if (opts->seconds)
      opts->seconds[sw] =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    report->sweeps = sw + 1;
    report->energy = e;
    report->alpha = alpha;
    const double rel = sw > 0 ? std::fabs(e - prev) / std::fabs(e) : INFINITY;
    prev = e;
    if (final_stage) {
      ++final_sweeps;
      if (final_sweeps >= 2 && rel < opts->conv_tol) {
        report->converged = 1;
        done = true;
      }
    } else {
      ++report->bulk_sweeps;
      if (rel < opts->switch_tol) {   // later sweeps in the final precision
        final_stage = true;
        uo.precision = opts->final_precision;
      }
    }
    if (++sw >= opts->max_sweeps) done = true;
  }
};
}  // namespace

extern "C" dmrg3s_status dmrg3s_sweep(dmrg3s_state state, const dmrg3s_alpha_rule* rule,
                                      const dmrg3s_sweep_opts* opts, double* energies,
                                      dmrg3s_sweep_report* report, dmrg3s_stream stream) {
  State* S = reinterpret_cast<State*>(state);
  if (!S || !rule || !opts || !report) return DMRG3S_ERR_ARG;
  Sweeper w;
  w.S = S;
  w.rule = rule;
  w.opts = opts;
  w.energies = energies;
  w.report = report;
  dmrg3s_status s = w.init(S->c);
  if (s) return s;
  while (!w.done) {
    dmrg3s_update_info inf{};
    if ((s = dmrg3s_local_update(state, w.dir(), w.alpha, &w.uo, &inf, stream))) return s;
    w.after(inf);
  }
  return DMRG3S_OK;
}

extern "C" dmrg3s_status dmrg3s_sweep_batch(const dmrg3s_state* states, int32_t nstates,
                                            const dmrg3s_alpha_rule* rules,
                                            const dmrg3s_sweep_opts* opts,
                                            double* const* energies, dmrg3s_sweep_report* reports,
                                            dmrg3s_stream stream) {
  Context* c = nullptr;
  dmrg3s_status s;
  if ((s = check_batch(states, nstates, &c))) return s;
  if (!rules || !opts || !reports) return fail(c, DMRG3S_ERR_ARG, "NULL argument");
  std::vector<Sweeper> sw(nstates);
  for (int k = 0; k < nstates; ++k) {
    sw[k].S = reinterpret_cast<State*>(states[k]);
    sw[k].rule = &rules[k];
    sw[k].opts = &opts[k];
    sw[k].energies = energies ? energies[k] : nullptr;
    sw[k].report = &reports[k];
    if ((s = sw[k].init(c))) return s;
    if (opts[k].update.svd != opts[0].update.svd)
      return fail(c, DMRG3S_ERR_ARG, "the states of a batch use one SVD method");
  }
  if ((s = use_device(c))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (;;) {
    std::vector<BItem> items;
    std::vector<int> who;
    for (int k = 0; k < nstates; ++k) {
      if (sw[k].done) continue;
      BItem it;
      if ((s = make_opts(c, sw[k].dir(), &sw[k].uo, &it.o))) return s;
      it.S = sw[k].S;
      it.dir = sw[k].dir();
      it.alpha = sw[k].alpha;
      items.push_back(std::move(it));
      who.push_back(k);
    }
    if (items.empty()) break;
    if ((s = local_update_batch(c, items, opts[0].update.svd, st))) return s;
    for (size_t j = 0; j < items.size(); ++j) {
      dmrg3s_update_info inf{};
      report_info(items[j].S, items[j].info, &inf);
      sw[who[j]].after(inf);
    }
  }
  return DMRG3S_OK;
}
