// Host-side planning of the block-sparse contractions.  See plan.hpp.
#include "plan.hpp"

#include "validate.hpp"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <map>
#include <set>

namespace dmrg3s {

void GemmStage::add(int64_t offC, int ldc, int M, int N, const std::vector<GemmSeg>& s) {
  if (M <= 0 || N <= 0) return;
  GemmTask t{};
  t.offC = offC;
  t.ldc = ldc;
  t.M = M;
  t.N = N;
  t.seg0 = (int32_t)segs.size();
  t.nseg = (int32_t)s.size();
  const int id = (int)tasks.size();
  tasks.push_back(t);
  for (const auto& g : s) {
    segs.push_back(g);
    flops += 2.0 * M * (double)N * g.K;
  }
  const int ntm = (M + 63) / 64, ntn = (N + 63) / 64;
  for (int a = 0; a < ntm; ++a)
    for (int b = 0; b < ntn; ++b) tiles.push_back(GemmTile{id, a, b, 0});
}

void GemmStage::finalize_bytes(Trans, Trans) {
  std::set<std::pair<int64_t, int64_t>> a, b;
  double elems = 0.0;
  for (const GemmTask& t : tasks) {
    elems += (double)t.M * t.N;
    for (int k = 0; k < t.nseg; ++k) {
      const GemmSeg& g = segs[t.seg0 + k];
      a.insert({g.offA, (int64_t)t.M * g.K});
      b.insert({g.offB, (int64_t)t.N * g.K});
    }
  }
  for (auto& x : a) elems += (double)x.second;
  for (auto& x : b) elems += (double)x.second;
  bytes = 8.0 * elems;
}

void CombStage::add(int64_t offOut, int ldo, int rows, int cols, const std::vector<CombTerm>& t) {
  if (rows <= 0 || cols <= 0) return;
  CombTask task{};
  task.offOut = offOut;
  task.ldo = ldo;
  task.rows = rows;
  task.cols = cols;
  task.t0 = (int32_t)terms.size();
  task.nt = (int32_t)t.size();
  const int id = (int)tasks.size();
  tasks.push_back(task);
  for (CombTerm tm : t) {
    tm.chi = (float)tm.coef;
    tm.clo = (float)(tm.coef - (double)tm.chi);
    terms.push_back(tm);
  }
  flops += 2.0 * rows * (double)cols * t.size();
  bytes += 8.0 * rows * (double)cols * (1 + t.size());
  for (int r = 0; r < rows; r += kCombRows)
    chunks.push_back(CombChunk{id, r, rows - r < kCombRows ? rows - r : kCombRows, 0});
}

namespace {
std::atomic<int> g_plan_ctas{152};
}  // namespace

void set_plan_ctas(int n) {
  if (n > 0 && n <= 4096) g_plan_ctas.store(n);
}
int plan_ctas() { return g_plan_ctas.load(); }

namespace {

// Static schedule of a stage's units over the persistent CTAs: longest
// processing time first onto the least loaded CTA.  A unit's cost is its
// k-chunks, each weighted 0.7 as a fixed share (the A slab's copy and the
// issue latency, the same for every width) and 0.3 by its MMA width, plus a
// fixed share for its drain and store.
void schedule_units(TcStage& tc, const std::vector<GemmTask>& tasks) {
  const int n = (int)tc.units.size();
  const int nc = std::max(1, std::min(plan_ctas(), n));
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    const TcUnit& u = tc.units[i];
    const int nrem = std::min(128, tasks[u.task].N - u.tn * 128);
    cost[i] = u.nchunks * (0.7 + 0.3 * (double)((nrem + 15) / 16 * 16) / 128.0) + 4.0;
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> lists(nc);
  std::vector<double> load(nc, 0.0);
  for (int i : order) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lists[c].push_back(i);
    load[c] += cost[i];
  }
  std::vector<TcUnit> out;
  out.reserve(n);
  tc.cta_start.assign(nc + 1, 0);
  for (int c = 0; c < nc; ++c) {
    tc.cta_start[c] = (int32_t)out.size();
    for (int i : lists[c]) out.push_back(tc.units[i]);
  }
  tc.cta_start[nc] = (int32_t)out.size();
  tc.units.swap(out);
}

using Key = std::array<int, 4>;
struct Interm {
  int64_t off;
  int rows, cols;
};
struct Combo {
  int rows = 0, cols = 0;
  std::vector<CombTerm> terms;
};

inline GemmSeg seg(int64_t offA, int64_t lda, int64_t offB, int64_t ldb, int64_t K) {
  GemmSeg g{};
  g.offA = offA;
  g.offB = offB;
  g.lda = (int32_t)lda;
  g.ldb = (int32_t)ldb;
  g.K = (int32_t)K;
  g.scale = 1.0;
  return g;
}

// Stage 1 + 2 of the left side: T1[bl, s] = L[bl] M[s]; T2 terms.
void left_stages(const EnvLayout& le, const MpoLayout& W, const SiteLayout& M, Plan* p,
                 std::map<Key, Interm>* t1, std::map<Key, Combo>* t2) {
  p->g1.ta = Trans::N;
  p->g1.tb = Trans::N;
  int64_t off = 0;
  for (const Block& lb : le.blocks) {
    const int bl = lb.a, ip = lb.b, i = lb.c;
    for (int s = 0; s < M.d; ++s) {
      const int mb = M.block_of(s, i);
      if (mb < 0) continue;
      const Block& blk = M.blocks[mb];
      const int j = blk.c;
      const int64_t rows = le.bond.dim[ip], cols = M.right.dim[j], K = M.left.dim[i];
      (*t1)[Key{bl, s, i, 0}] = Interm{off, (int)rows, (int)cols};
      p->g1.add(off, (int)cols, (int)rows, (int)cols, {seg(lb.off, K, blk.off, cols, K)});
      // stage 2 terms
      for (int so = 0; so < W.d; ++so)
        for (int br = 0; br < W.wr; ++br) {
          const double c = W.at(so, s, bl, br);
          if (c == 0.0) continue;
          Combo& cb = (*t2)[Key{br, so, ip, j}];
          cb.rows = (int)rows;
          cb.cols = (int)cols;
          CombTerm tm{};
          tm.offIn = off;
          tm.ldi = (int32_t)cols;
          tm.coef = c;
          cb.terms.push_back(tm);
        }
      off += rows * cols;
    }
  }
  p->ws1 = off;
}

// Stage 1 + 2 of the right side: U1[br, s] = M[s] R[br]^T; U2 terms.
void right_stages(const EnvLayout& re, const MpoLayout& W, const SiteLayout& M, Plan* p,
                  std::map<Key, Interm>* u1, std::map<Key, Combo>* u2) {
  p->g1.ta = Trans::N;
  p->g1.tb = Trans::T;
  int64_t off = 0;
  for (const Block& mb : M.blocks) {
    const int s = mb.a, i = mb.b, j = mb.c;
    for (int br = 0; br < re.w; ++br) {
      const int rb = re.block_of(br, j);
      if (rb < 0) continue;
      const Block& rblk = re.blocks[rb];
      const int jp = rblk.b;
      const int64_t rows = M.left.dim[i], cols = re.bond.dim[jp], K = M.right.dim[j];
      (*u1)[Key{br, s, i, 0}] = Interm{off, (int)rows, (int)cols};
      p->g1.add(off, (int)cols, (int)rows, (int)cols, {seg(mb.off, K, rblk.off, K, K)});
      for (int so = 0; so < W.d; ++so)
        for (int bl = 0; bl < W.wl; ++bl) {
          const double c = W.at(so, s, bl, br);
          if (c == 0.0) continue;
          Combo& cb = (*u2)[Key{bl, so, i, jp}];
          cb.rows = (int)rows;
          cb.cols = (int)cols;
          CombTerm tm{};
          tm.offIn = off;
          tm.ldi = (int32_t)cols;
          tm.coef = c;
          cb.terms.push_back(tm);
        }
      off += rows * cols;
    }
  }
  p->ws1 = off;
}

// Materialise stage-2 blocks contiguously in ws2 (offsets in map order).
std::map<Key, Interm> materialise(const std::map<Key, Combo>& combos, Plan* p) {
  std::map<Key, Interm> out;
  int64_t off = 0;
  for (const auto& kv : combos) {
    const Combo& cb = kv.second;
    out[kv.first] = Interm{off, cb.rows, cb.cols};
    p->c2.add(off, cb.cols, cb.rows, cb.cols, cb.terms);
    off += (int64_t)cb.rows * cb.cols;
  }
  p->ws2 = off;
  return out;
}

// ---- tensor-core form of the stages ----

inline int32_t groups8(int64_t R) { return (int32_t)((R + 7) / 8); }
inline int32_t chunks32(int64_t K) { return (int32_t)((K + 31) / 32); }

// Packed placements of one operand array; identical views share one block.
struct Packer {
  std::map<std::pair<std::array<int64_t, 5>, double>, int64_t> seen;   // (view, scale) -> dst
  std::vector<PackBlock>* out;
  int64_t* n;
  int32_t* tiles;
  int64_t add(int64_t src, int64_t ld, int64_t R, int64_t K, int trans, double scale = 1.0) {
    const auto key = std::make_pair(std::array<int64_t, 5>{src, ld, R, K, trans}, scale);
    auto it = seen.find(key);
    if (it != seen.end()) return it->second;
    PackBlock b{};
    b.src = src;
    b.scale = scale;
    int ex = 0;
    b.pow2 = (std::frexp(scale, &ex) == 0.5 || std::frexp(scale, &ex) == -0.5) && ex > -100 && ex < 100
                 ? (float)scale
                 : 0.f;
    b.dst = *n;
    b.ld = (int32_t)ld;
    b.R = (int32_t)R;
    b.K = (int32_t)K;
    b.trans = trans;
    b.R8 = groups8(R);
    b.KC = chunks32(K);
    b.tile0 = *tiles;
    out->push_back(b);
    *n += (int64_t)b.R8 * b.KC * kPackTile;
    *tiles += b.R8 * b.KC;
    seen[key] = b.dst;
    return b.dst;
  }
};

// Placement of a block packed by stage 2: ws2 element offset -> (dst, R8, R, K).
struct CombPacked {
  int64_t dst;
  int32_t R8, R, K;
};

// Builds g.tc.  An operand with a map (c2A for A, c2B for B) is the stage-2
// output, already packed; its segments look their block up by the ws2 offset.
bool build_tc(GemmStage& g, const std::map<int64_t, CombPacked>* c2A,
              const std::map<int64_t, CombPacked>* c2B, std::string* err) {
  TcStage& tc = g.tc;
  tc = TcStage();
  Packer pa{{}, &tc.packA, &tc.nA, &tc.tilesA};
  Packer pb{{}, &tc.packB, &tc.nB, &tc.tilesB};
  auto lookup = [&](const std::map<int64_t, CombPacked>* m, int64_t off, int64_t R, int64_t K,
                    int64_t* dst, int32_t* r8) {
    auto it = m->find(off);
    if (it == m->end() || it->second.R != R || it->second.K != K) {
      *err = "tensor-core operand of stage 3 is not a stage-2 block";
      return false;
    }
    *dst = it->second.dst;
    *r8 = it->second.R8;
    return true;
  };
  for (const GemmTask& t : g.tasks) {
    int32_t nch = 0;
    for (int k = 0; k < t.nseg; ++k) {
      const GemmSeg& sg = g.segs[t.seg0 + k];
      TcSeg ts{};
      ts.kc = chunks32(sg.K);
      // A (rows M): ta = N stores M x K, ta = T stores K x M
      if (c2A) {
        if (!lookup(c2A, sg.offA, t.M, sg.K, &ts.pa, &ts.ra8)) return false;
      } else {
        ts.pa = pa.add(sg.offA, sg.lda, t.M, sg.K, g.ta == Trans::T ? 1 : 0);
        ts.ra8 = groups8(t.M);
      }
      // B (rows N): tb = N stores K x N, tb = T stores N x K
      if (c2B) {
        if (!lookup(c2B, sg.offB, t.N, sg.K, &ts.pb, &ts.rb8)) return false;
      } else {
        ts.pb = pb.add(sg.offB, sg.ldb, t.N, sg.K, g.tb == Trans::N ? 1 : 0);
        ts.rb8 = groups8(t.N);
      }
      tc.segs.push_back(ts);
      nch += ts.kc;
    }
    const int id = (int)(&t - g.tasks.data());
    for (int a = 0; a < (t.M + 127) / 128; ++a)
      for (int b = 0; b < (t.N + 127) / 128; ++b) tc.units.push_back(TcUnit{id, a, b, nch});
  }
  schedule_units(tc, g.tasks);
  return true;
}

// Packs every stage-2 output block (orientation `trans`) and returns the map
// from its ws2 offset to the packed placement.
std::map<int64_t, CombPacked> pack_c2(Plan* p, int trans) {
  std::map<int64_t, CombPacked> m;
  p->c2pack.clear();
  p->nT2p = 0;
  p->tilesT2 = 0;
  for (const CombTask& t : p->c2.tasks) {
    PackOut o{};
    const int64_t R = trans ? t.cols : t.rows, K = trans ? t.rows : t.cols;
    o.dst = p->nT2p;
    o.R8 = groups8(R);
    o.KC = chunks32(K);
    o.trans = trans;
    o.tile0 = p->tilesT2;
    p->c2pack.push_back(o);
    m[t.offOut] = CombPacked{o.dst, o.R8, (int32_t)R, (int32_t)K};
    p->nT2p += (int64_t)o.R8 * o.KC * kPackTile;
    p->tilesT2 += o.R8 * o.KC;
  }
  return m;
}

// Units per GPU the split-K grouping of stage 3 aims at (two per SM of a GB300).
constexpr int64_t kTargetUnits = 2 * 152;

// The fused stages 1 + 2 of H_eff: one task per stage-2 block T2 (packed
// output at its c2pack placement), one K-segment per MPO term of that block:
// A = coef * L[bl] (the stage-1 A operand of the term's T1 block), B = M[s].
bool build_fused(Plan* p, const std::map<int64_t, CombPacked>& c2p, std::string* err) {
  std::map<int64_t, int> t1_task;      // T1 element offset -> stage-1 task
  for (size_t i = 0; i < p->g1.tasks.size(); ++i) t1_task[p->g1.tasks[i].offC] = (int)i;
  GemmStage& g = p->g12;
  g = GemmStage();
  g.ta = p->g1.ta;
  g.tb = p->g1.tb;
  TcStage& tc = g.tc;
  Packer pa{{}, &tc.packA, &tc.nA, &tc.tilesA};
  Packer pb{{}, &tc.packB, &tc.nB, &tc.tilesB};
  for (const CombTask& ct : p->c2.tasks) {
    auto it = c2p.find(ct.offOut);
    if (it == c2p.end()) {
      *err = "fused stage: stage-2 block without a packed placement";
      return false;
    }
    GemmTask t{};
    t.offC = it->second.dst;
    t.ldc = it->second.R8;
    t.M = ct.rows;
    t.N = ct.cols;
    t.seg0 = (int32_t)g.segs.size();
    t.nseg = ct.nt;
    int32_t nch = 0;
    for (int k = 0; k < ct.nt; ++k) {
      const CombTerm& tm = p->c2.terms[ct.t0 + k];
      auto jt = t1_task.find(tm.offIn);
      if (jt == t1_task.end()) {
        *err = "fused stage: MPO term without a stage-1 block";
        return false;
      }
      const GemmTask& t1 = p->g1.tasks[jt->second];
      if (t1.nseg != 1 || t1.M != ct.rows || t1.N != ct.cols) {
        *err = "fused stage: stage-1 block shape";
        return false;
      }
      const GemmSeg& s1 = p->g1.segs[t1.seg0];
      g.segs.push_back(s1);
      TcSeg ts{};
      ts.kc = chunks32(s1.K);
      ts.pa = pa.add(s1.offA, s1.lda, t.M, s1.K, g.ta == Trans::T ? 1 : 0, tm.coef);
      ts.ra8 = groups8(t.M);
      ts.pb = pb.add(s1.offB, s1.ldb, t.N, s1.K, g.tb == Trans::N ? 1 : 0);
      ts.rb8 = groups8(t.N);
      tc.segs.push_back(ts);
      nch += ts.kc;
    }
    const int id = (int)g.tasks.size();
    g.tasks.push_back(t);
    for (int a = 0; a < (t.M + 127) / 128; ++a)
      for (int b = 0; b < (t.N + 127) / 128; ++b) tc.units.push_back(TcUnit{id, a, b, nch});
  }
  schedule_units(tc, g.tasks);
  // algorithmic work: that of stages 1 and 2, which this stage replaces
  g.flops = p->g1.flops + p->c2.flops;
  g.bytes = p->g1.bytes + p->c2.bytes;
  p->fused = true;
  return true;
}

// Smaller combination chunks when a stage would have fewer than `target`
// of them (small blocks: more CTAs, each with fewer rows).
void rechunk(CombStage& c, int target) {
  int rpc = kCombRows;
  auto count = [&](int r) {
    int64_t n = 0;
    for (const CombTask& t : c.tasks) n += (t.rows + r - 1) / r;
    return n;
  };
  while (rpc > 1 && count(rpc) < target) rpc /= 2;
  if (rpc == kCombRows) return;
  c.chunks.clear();
  for (size_t id = 0; id < c.tasks.size(); ++id) {
    const int rows = c.tasks[id].rows;
    for (int r = 0; r < rows; r += rpc)
      c.chunks.push_back(CombChunk{(int32_t)id, r, rows - r < rpc ? rows - r : rpc, 0});
  }
}

// Bounds of every table against the buffers the stages address.
dmrg3s_status finish(Plan* p, int64_t nA1, int64_t nB1, int64_t nOut2, int64_t nA3, int64_t nB3,
                     int64_t nC3, std::string* err) {
  p->nA1 = nA1;
  p->nB1 = nB1;
  p->nA3 = p->has_g3 ? nA3 : 0;
  p->nB3 = p->has_g3 ? nB3 : 0;
  p->g1.finalize_bytes(p->g1.ta, p->g1.tb);
  if (p->has_g3) p->g3.finalize_bytes(p->g3.ta, p->g3.tb);
  if (p->has_g3) {
    // split-K form of stage 3: the K-segments of every output block in G
    // consecutive groups, G chosen so that the units fill the GPU about twice
    // (kTargetUnits); each group writes a partial block, then a fixed-order sum
    int64_t units1 = 0;
    int maxseg = 1;
    for (const GemmTask& t : p->g3.tasks) {
      units1 += (int64_t)((t.M + 127) / 128) * ((t.N + 127) / 128);
      maxseg = std::max(maxseg, (int)t.nseg);
    }
    int G = units1 > 0 ? (int)((kTargetUnits + units1 - 1) / units1) : 1;
    G = std::max(1, std::min(G, maxseg));
    p->g3s.ta = p->g3.ta;
    p->g3s.tb = p->g3.tb;
    int64_t poff = 0;
    for (const GemmTask& t : p->g3.tasks) {
      std::vector<CombTerm> terms;
      const int ng = std::min<int>(G, std::max(1, (int)t.nseg));
      for (int gi = 0; gi < ng; ++gi) {
        const int k0 = (int)((int64_t)t.nseg * gi / ng), k1 = (int)((int64_t)t.nseg * (gi + 1) / ng);
        std::vector<GemmSeg> sg(p->g3.segs.begin() + t.seg0 + k0, p->g3.segs.begin() + t.seg0 + k1);
        if (sg.empty() && t.nseg > 0) continue;
        p->g3s.add(poff, t.N, t.M, t.N, sg);
        CombTerm tm{};
        tm.offIn = poff;
        tm.ldi = t.N;
        tm.coef = 1.0;
        terms.push_back(tm);
        poff += (int64_t)t.M * t.N;
      }
      p->c3r.add(t.offC, t.ldc, t.M, t.N, terms);
    }
    p->ws3 = poff;
    p->g3s.flops = p->g3.flops;        // same algorithmic work as stage 3
    p->g3s.bytes = p->g3.bytes;
    p->c3r.flops = 0.0;                // the partial sums are bookkeeping, not algorithm
    p->c3r.bytes = 0.0;
    const int64_t w3 = poff > 0 ? poff : 1;
    if (!gemm_ok(p->g3s.ta, p->g3s.tb, p->g3s.tasks, p->g3s.segs, nA3, nB3, w3, err) ||
        !comb_ok(p->c3r.tasks, p->c3r.terms, w3, nC3, err)) {
      *err = "internal planning error: " + *err;
      return DMRG3S_ERR_SHAPE;
    }
  }
  const int64_t w1 = p->ws1 > 0 ? p->ws1 : 1;
  if (!gemm_ok(p->g1.ta, p->g1.tb, p->g1.tasks, p->g1.segs, nA1, nB1, w1, err) ||
      !comb_ok(p->c2.tasks, p->c2.terms, w1, nOut2, err) ||
      (p->has_g3 && !gemm_ok(p->g3.ta, p->g3.tb, p->g3.tasks, p->g3.segs, nA3, nB3, nC3, err))) {
    *err = "internal planning error: " + *err;
    return DMRG3S_ERR_SHAPE;
  }
  // tensor-core form.  H_eff: stages 1 and 2 fused (g12) writing T2 packed
  // for stage 3.  The others: stage 1 packs both operands, and stage 3 takes
  // the stage-2 output packed by the combination (B of the environments).
  bool ok = true;
  if (p->kind == Kind::Heff) {
    const std::map<int64_t, CombPacked> m = pack_c2(p, 0);
    ok = build_fused(p, m, err) && build_tc(p->g3s, &m, nullptr, err) &&
         tc_ok(p->g12.tasks, p->g12.tc, nA1, nB1, p->g12.tc.nA, p->g12.tc.nB, err) &&
         packed_tasks_ok(p->g12.tasks, p->nT2p, err);
  } else {
    ok = build_tc(p->g1, nullptr, nullptr, err);
    if (ok && p->has_g3) {
      const int trans = p->kind == Kind::EnvLR ? 1 : 0;
      const std::map<int64_t, CombPacked> m = pack_c2(p, trans);
      ok = build_tc(p->g3s, nullptr, &m, err);
    }
    if (ok) ok = tc_ok(p->g1.tasks, p->g1.tc, nA1, nB1, p->g1.tc.nA, p->g1.tc.nB, err);
  }
  if (ok && p->has_g3) {
    const bool c2_is_a = p->kind == Kind::Heff;
    ok = tc_ok(p->g3s.tasks, p->g3s.tc, nA3, nB3, c2_is_a ? p->nT2p : p->g3s.tc.nA,
               c2_is_a ? p->g3s.tc.nB : p->nT2p, err) &&
         packout_ok(p->c2.tasks, p->c2pack, p->nT2p, err);
  }
  if (!ok) {
    *err = "internal planning error: " + *err;
    return DMRG3S_ERR_SHAPE;
  }
  rechunk(p->c2, 2 * plan_ctas());
  rechunk(p->c3r, 2 * plan_ctas());
  return DMRG3S_OK;
}

}  // namespace

namespace {
// Appends stage `src` to `dst` with its operand offsets moved by oA / oB and
// its output offsets by oC.
void append_gemm(GemmStage& dst, const GemmStage& src, int64_t oA, int64_t oB, int64_t oC) {
  const int32_t t0 = (int32_t)dst.tasks.size(), s0 = (int32_t)dst.segs.size();
  for (GemmTask t : src.tasks) {
    t.offC += oC;
    t.seg0 += s0;
    dst.tasks.push_back(t);
  }
  for (GemmSeg g : src.segs) {
    g.offA += oA;
    g.offB += oB;
    dst.segs.push_back(g);
  }
  for (GemmTile t : src.tiles) {
    t.task += t0;
    dst.tiles.push_back(t);
  }
  dst.flops += src.flops;
}
void append_comb(CombStage& dst, const CombStage& src, int64_t oIn, int64_t oOut, double scale) {
  const int32_t t0 = (int32_t)dst.tasks.size(), m0 = (int32_t)dst.terms.size();
  for (CombTask t : src.tasks) {
    t.offOut += oOut;
    t.t0 += m0;
    dst.tasks.push_back(t);
  }
  for (CombTerm m : src.terms) {
    m.offIn += oIn;
    if (scale != 1.0) {
      m.coef *= scale;
      m.chi = (float)m.coef;
      m.clo = (float)(m.coef - (double)m.chi);
    }
    dst.terms.push_back(m);
  }
  for (CombChunk ch : src.chunks) {
    ch.task += t0;
    dst.chunks.push_back(ch);
  }
  dst.flops += src.flops;
  dst.bytes += src.bytes;
}
}  // namespace

dmrg3s_status merge_plans(Kind kind, const std::vector<PlanPart>& parts, int64_t nA1, int64_t nB1,
                          int64_t nOut2, int64_t nA3, int64_t nB3, int64_t nC3, Plan* out,
                          std::string* err) {
  *out = Plan();
  Plan& m = *out;
  m.kind = kind;
  m.has_g3 = kind == Kind::Heff || kind == Kind::EnvLR || kind == Kind::EnvRL;
  if (parts.empty()) {
    *err = "merge of no plans";
    return DMRG3S_ERR_ARG;
  }
  m.g1.ta = parts[0].p->g1.ta;
  m.g1.tb = parts[0].p->g1.tb;
  m.g3.ta = parts[0].p->g3.ta;
  m.g3.tb = parts[0].p->g3.tb;
  int64_t o1 = 0, o2 = 0;
  for (const PlanPart& q : parts) {
    const Plan& p = *q.p;
    if (p.kind != kind || p.g1.ta != m.g1.ta || p.g1.tb != m.g1.tb ||
        (m.has_g3 && (p.g3.ta != m.g3.ta || p.g3.tb != m.g3.tb))) {
      *err = "merged plans differ in kind";
      return DMRG3S_ERR_ARG;
    }
    append_gemm(m.g1, p.g1, q.oA1, q.oB1, o1);
    append_comb(m.c2, p.c2, o1, m.has_g3 ? o2 : q.oOut2, q.c2scale);
    if (m.has_g3) {
      const bool t2_is_a = kind == Kind::Heff;
      append_gemm(m.g3, p.g3, t2_is_a ? o2 : q.oA3, t2_is_a ? q.oB3 : o2, q.oC3);
    }
    o1 += p.ws1;
    o2 += m.has_g3 ? p.ws2 : 0;
  }
  m.ws1 = o1;
  m.ws2 = o2;
  if (m.has_g3) {
    if (kind == Kind::Heff) nA3 = o2;
    else nB3 = o2;
    nOut2 = o2;
  }
  return finish(&m, nA1, nB1, nOut2, nA3, nB3, nC3, err);
}

dmrg3s_status check_site_mpo(const SiteLayout& s, const MpoLayout& W, std::string* err) {
  if (s.nsym != W.nsym) {
    *err = "site tensor and MPO have different nsym";
    return DMRG3S_ERR_SHAPE;
  }
  if (s.d != W.d) {
    *err = "site tensor and MPO have different physical dimension";
    return DMRG3S_ERR_SHAPE;
  }
  if (!same_charges(s.qp, W.qp)) {
    *err = "site tensor and MPO have different physical charges";
    return DMRG3S_ERR_QN;
  }
  return DMRG3S_OK;
}

dmrg3s_status check_env(const EnvLayout& e, const Bond& bond, int w, const std::vector<Charge>& t,
                        const char* what, std::string* err) {
  if (e.nsym != bond.nsym) {
    *err = std::string(what) + ": nsym differs from the site tensor";
    return DMRG3S_ERR_SHAPE;
  }
  if (!same_bond(e.bond, bond)) {
    *err = std::string(what) + ": bond differs from the site tensor's bond";
    return DMRG3S_ERR_SHAPE;
  }
  if (e.w != w) {
    *err = std::string(what) + ": MPO bond dimension differs from W";
    return DMRG3S_ERR_SHAPE;
  }
  if (!same_charges(e.t, t)) {
    *err = std::string(what) + ": channel charges differ from W";
    return DMRG3S_ERR_QN;
  }
  return DMRG3S_OK;
}

dmrg3s_status plan_heff(const EnvLayout& le, const MpoLayout& W, const EnvLayout& re,
                        const SiteLayout& M, Plan* p, std::string* err) {
  p->kind = Kind::Heff;
  std::map<Key, Interm> t1;
  std::map<Key, Combo> t2c;
  left_stages(le, W, M, p, &t1, &t2c);
  std::map<Key, Interm> t2 = materialise(t2c, p);
  p->has_g3 = true;
  p->g3.ta = Trans::N;
  p->g3.tb = Trans::T;
  for (const Block& hb : M.blocks) {
    const int so = hb.a, ip = hb.b, jp = hb.c;
    std::vector<GemmSeg> segs;
    for (int br = 0; br < W.wr; ++br) {
      const int j = M.nsym ? M.right.find(sub(M.right.q[jp], re.t[br])) : 0;
      if (j < 0) continue;
      const int rb = re.block_of(br, j);
      if (rb < 0 || re.blocks[rb].b != jp) continue;
      auto it = t2.find(Key{br, so, ip, j});
      if (it == t2.end()) continue;
      const int64_t K = M.right.dim[j];
      segs.push_back(seg(it->second.off, K, re.blocks[rb].off, K, K));
    }
    p->g3.add(hb.off, (int)hb.cols, (int)hb.rows, (int)hb.cols, segs);
  }
  return finish(p, le.size, M.size, p->ws2, p->ws2, re.size, M.size, err);
}

dmrg3s_status plan_expand_lr(const EnvLayout& le, const MpoLayout& W, const SiteLayout& M,
                             const SiteLayout& P, const FusedBond& fused, Plan* p,
                             std::string* err) {
  p->kind = Kind::ExpandLR;
  std::map<Key, Interm> t1;
  std::map<Key, Combo> t2c;
  left_stages(le, W, M, p, &t1, &t2c);
  const int nsrc = M.right.nsec();
  for (const Block& pb : P.blocks) {
    const int so = pb.a, ip = pb.b, k = pb.c;
    for (int br = 0; br < W.wr; ++br) {
      const int j = M.nsym ? M.right.find(sub(P.right.q[k], W.tr[br])) : 0;
      if (j < 0 || fused.target[(size_t)br * nsrc + j] != k) continue;
      const int64_t coff = fused.offset[(size_t)br * nsrc + j];
      auto it = t2c.find(Key{br, so, ip, j});
      static const std::vector<CombTerm> none;
      p->c2.add(pb.off + coff, (int)pb.cols, (int)pb.rows, (int)M.right.dim[j],
                it == t2c.end() ? none : it->second.terms);
    }
  }
  p->ws2 = 0;
  return finish(p, le.size, M.size, P.size, 0, 0, 0, err);
}

dmrg3s_status plan_env_lr(const EnvLayout& le, const MpoLayout& W, const SiteLayout& M,
                          const EnvLayout& out, Plan* p, std::string* err) {
  p->kind = Kind::EnvLR;
  std::map<Key, Interm> t1;
  std::map<Key, Combo> t2c;
  left_stages(le, W, M, p, &t1, &t2c);
  std::map<Key, Interm> t2 = materialise(t2c, p);
  p->has_g3 = true;
  p->g3.ta = Trans::T;
  p->g3.tb = Trans::N;
  for (const Block& ob : out.blocks) {
    const int br = ob.a, ib = ob.b, ik = ob.c;
    std::vector<GemmSeg> segs;
    for (int so = 0; so < M.d; ++so) {
      const int ip = M.nsym ? M.left.find(sub(M.right.q[ib], M.qp[so])) : 0;
      if (ip < 0) continue;
      const int ab = M.block_of(so, ip);
      if (ab < 0 || M.blocks[ab].c != ib) continue;
      auto it = t2.find(Key{br, so, ip, ik});
      if (it == t2.end()) continue;
      const int64_t K = M.left.dim[ip];
      segs.push_back(seg(M.blocks[ab].off, M.right.dim[ib], it->second.off, M.right.dim[ik], K));
    }
    p->g3.add(ob.off, (int)ob.cols, (int)ob.rows, (int)ob.cols, segs);
  }
  return finish(p, le.size, M.size, p->ws2, M.size, p->ws2, out.size, err);
}

dmrg3s_status plan_expand_rl(const EnvLayout& re, const MpoLayout& W, const SiteLayout& M,
                             const SiteLayout& P, const FusedBond& fused, Plan* p,
                             std::string* err) {
  p->kind = Kind::ExpandRL;
  std::map<Key, Interm> u1;
  std::map<Key, Combo> u2c;
  right_stages(re, W, M, p, &u1, &u2c);
  const int nsrc = M.left.nsec();
  for (const Block& pb : P.blocks) {
    const int so = pb.a, k = pb.b, jp = pb.c;
    for (int bl = 0; bl < W.wl; ++bl) {
      const int i = M.nsym ? M.left.find(sub(P.left.q[k], W.tl[bl])) : 0;
      if (i < 0 || fused.target[(size_t)bl * nsrc + i] != k) continue;
      const int64_t roff = fused.offset[(size_t)bl * nsrc + i];
      auto it = u2c.find(Key{bl, so, i, jp});
      static const std::vector<CombTerm> none;
      p->c2.add(pb.off + roff * pb.cols, (int)pb.cols, (int)M.left.dim[i], (int)pb.cols,
                it == u2c.end() ? none : it->second.terms);
    }
  }
  p->ws2 = 0;
  return finish(p, M.size, re.size, P.size, 0, 0, 0, err);
}

dmrg3s_status plan_env_rl(const EnvLayout& re, const MpoLayout& W, const SiteLayout& M,
                          const EnvLayout& out, Plan* p, std::string* err) {
  p->kind = Kind::EnvRL;
  std::map<Key, Interm> u1;
  std::map<Key, Combo> u2c;
  right_stages(re, W, M, p, &u1, &u2c);
  std::map<Key, Interm> u2 = materialise(u2c, p);
  p->has_g3 = true;
  p->g3.ta = Trans::N;
  p->g3.tb = Trans::T;
  for (const Block& ob : out.blocks) {
    const int bl = ob.a, ib = ob.b, ik = ob.c;
    std::vector<GemmSeg> segs;
    for (int so = 0; so < M.d; ++so) {
      const int bb = M.block_of(so, ib);
      if (bb < 0) continue;
      const int jp = M.blocks[bb].c;
      auto it = u2.find(Key{bl, so, ik, jp});
      if (it == u2.end()) continue;
      const int64_t K = M.right.dim[jp];
      segs.push_back(seg(M.blocks[bb].off, K, it->second.off, K, K));
    }
    p->g3.add(ob.off, (int)ob.cols, (int)ob.rows, (int)ob.cols, segs);
  }
  return finish(p, M.size, re.size, p->ws2, M.size, p->ws2, out.size, err);
}

dmrg3s_status plan_mpo_grad(const EnvLayout& le, const MpoLayout& W, const EnvLayout& re,
                            const SiteLayout& M, GradPlan* p, std::string* err) {
  // stage 1 exactly as for H_eff; the T1 blocks are then indexed by (bl, s)
  Plan tmp;
  std::map<Key, Interm> t1;
  std::map<Key, Combo> unused;
  left_stages(le, W, M, &tmp, &t1, &unused);
  p->g1 = tmp.g1;
  p->ws1 = tmp.ws1;
  struct T1Blk {
    int ip, j;
    int64_t off, len;
  };
  std::map<std::pair<int, int>, std::vector<T1Blk>> by_bl_s;
  for (const auto& kv : t1) {
    const int bl = kv.first[0], s = kv.first[1], i = kv.first[2];
    const int lb = le.block_of(bl, i), mb = M.block_of(s, i);
    if (lb < 0 || mb < 0) continue;
    by_bl_s[{bl, s}].push_back(T1Blk{le.blocks[lb].b, M.blocks[mb].c, kv.second.off,
                                     (int64_t)kv.second.rows * kv.second.cols});
  }
  // Y[br, s'](al', ar) = M[s'](al', ar') R[br](ar', ar)
  p->gy.ta = Trans::N;
  p->gy.tb = Trans::N;
  std::map<Key, Interm> y;
  int64_t off = 0;
  for (const Block& mb : M.blocks) {
    const int so = mb.a, ip = mb.b, jp = mb.c;
    for (int br = 0; br < W.wr; ++br) {
      const int j = M.nsym ? M.right.find(sub(M.right.q[jp], re.t[br])) : 0;
      if (j < 0) continue;
      const int rb = re.block_of(br, j);
      if (rb < 0 || re.blocks[rb].b != jp) continue;
      const int64_t rows = M.left.dim[ip], cols = M.right.dim[j], K = M.right.dim[jp];
      y[Key{br, so, ip, j}] = Interm{off, (int)rows, (int)cols};
      p->gy.add(off, (int)cols, (int)rows, (int)cols, {seg(mb.off, K, re.blocks[rb].off, cols, K)});
      off += rows * cols;
    }
  }
  p->wsy = off;
  p->nG = (int64_t)W.d * W.d * W.wl * W.wr;
  for (int so = 0; so < W.d; ++so)
    for (int s = 0; s < W.d; ++s)
      for (int bl = 0; bl < W.wl; ++bl)
        for (int br = 0; br < W.wr; ++br) {
          DotTask t{};
          t.out = (((int64_t)so * W.d + s) * W.wl + bl) * W.wr + br;
          t.seg0 = (int32_t)p->segs.size();
          auto it = by_bl_s.find({bl, s});
          if (it != by_bl_s.end())
            for (const T1Blk& b : it->second) {
              auto yt = y.find(Key{br, so, b.ip, b.j});
              if (yt == y.end()) continue;
              p->segs.push_back(DotSeg{b.off, yt->second.off, b.len});
              p->dot_flops += 2.0 * b.len;
            }
          t.nseg = (int32_t)p->segs.size() - t.seg0;
          p->tasks.push_back(t);
        }
  p->g1.finalize_bytes(p->g1.ta, p->g1.tb);
  p->gy.finalize_bytes(p->gy.ta, p->gy.tb);
  const int64_t w1 = p->ws1 > 0 ? p->ws1 : 1, wy = p->wsy > 0 ? p->wsy : 1;
  if (!gemm_ok(p->g1.ta, p->g1.tb, p->g1.tasks, p->g1.segs, le.size, M.size, w1, err) ||
      !gemm_ok(p->gy.ta, p->gy.tb, p->gy.tasks, p->gy.segs, M.size, re.size, wy, err)) {
    *err = "internal planning error: " + *err;
    return DMRG3S_ERR_SHAPE;
  }
  for (const DotSeg& g : p->segs)
    if (g.offA < 0 || g.offB < 0 || g.len < 0 || g.offA + g.len > p->ws1 ||
        g.offB + g.len > p->wsy) {
      *err = "internal planning error: gradient segment out of bounds";
      return DMRG3S_ERR_SHAPE;
    }
  return DMRG3S_OK;
}

}  // namespace dmrg3s
