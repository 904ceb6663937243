// Host-side bounds validation of task tables before any launch: every element
// a kernel will read or write must lie inside the buffer it addresses.  A
// violation is an internal planning error and is reported as a status, so a
// bad table never reaches the device.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kernels.hpp"
#include "plan.hpp"
#include "vecops.hpp"

namespace dmrg3s {

inline bool span_ok(int64_t off, int64_t last, int64_t n) { return off >= 0 && off + last < n; }

inline bool gemm_ok(Trans ta, Trans tb, const std::vector<GemmTask>& tasks,
                    const std::vector<GemmSeg>& segs, int64_t nA, int64_t nB, int64_t nC,
                    std::string* err) {
  for (const GemmTask& t : tasks) {
    if (t.M <= 0 || t.N <= 0) continue;
    if (!span_ok(t.offC, (int64_t)(t.M - 1) * t.ldc + t.N - 1, nC) || t.ldc < t.N) {
      *err = "GEMM output out of bounds";
      return false;
    }
    for (int k = 0; k < t.nseg; ++k) {
      const GemmSeg& s = segs[t.seg0 + k];
      if (s.K <= 0) continue;
      const int64_t la = ta == Trans::N ? (int64_t)(t.M - 1) * s.lda + s.K - 1
                                        : (int64_t)(s.K - 1) * s.lda + t.M - 1;
      const int64_t lb = tb == Trans::N ? (int64_t)(s.K - 1) * s.ldb + t.N - 1
                                        : (int64_t)(t.N - 1) * s.ldb + s.K - 1;
      if (!span_ok(s.offA, la, nA) || !span_ok(s.offB, lb, nB)) {
        *err = "GEMM operand out of bounds";
        return false;
      }
    }
  }
  return true;
}

inline bool comb_ok(const std::vector<CombTask>& tasks, const std::vector<CombTerm>& terms,
                    int64_t nIn, int64_t nOut, std::string* err) {
  for (const CombTask& t : tasks) {
    if (t.rows <= 0 || t.cols <= 0) continue;
    if (!span_ok(t.offOut, (int64_t)(t.rows - 1) * t.ldo + t.cols - 1, nOut) || t.ldo < t.cols) {
      *err = "combination output out of bounds";
      return false;
    }
    for (int k = 0; k < t.nt; ++k) {
      const CombTerm& m = terms[t.t0 + k];
      if (!span_ok(m.offIn, (int64_t)(t.rows - 1) * m.ldi + t.cols - 1, nIn)) {
        *err = "combination input out of bounds";
        return false;
      }
    }
  }
  return true;
}

// Tensor-core tables: every packed source view inside its FP64 array, every
// packed block and every bulk copy of a unit inside its packed array.
inline bool pack_ok(const std::vector<PackBlock>& blocks, int64_t nSrc, int64_t nPacked,
                    int32_t ntiles, std::string* err) {
  for (const PackBlock& b : blocks) {
    if (b.R <= 0 || b.K <= 0) continue;
    const int64_t last = b.trans ? (int64_t)(b.K - 1) * b.ld + b.R - 1
                                 : (int64_t)(b.R - 1) * b.ld + b.K - 1;
    const int64_t minld = b.trans ? b.R : b.K;
    if (!span_ok(b.src, last, nSrc) || b.ld < minld || (int64_t)b.R8 * 8 < b.R ||
        (int64_t)b.KC * 32 < b.K || b.dst < 0 ||
        b.dst + (int64_t)b.R8 * b.KC * kPackTile > nPacked || b.tile0 < 0 ||
        (int64_t)b.tile0 + (int64_t)b.R8 * b.KC > ntiles) {
      *err = "operand pack out of bounds";
      return false;
    }
  }
  return true;
}

inline bool tc_ok(const std::vector<GemmTask>& tasks, const TcStage& tc, int64_t nSrcA,
                  int64_t nSrcB, int64_t nPA, int64_t nPB, std::string* err) {
  if (!pack_ok(tc.packA, nSrcA, tc.nA, tc.tilesA, err) ||
      !pack_ok(tc.packB, nSrcB, tc.nB, tc.tilesB, err))
    return false;
  std::vector<int32_t> nch(tasks.size(), 0);
  for (size_t i = 0; i < tasks.size(); ++i) {
    const GemmTask& t = tasks[i];
    if (t.seg0 < 0 || (size_t)t.seg0 + t.nseg > tc.segs.size()) {
      *err = "tensor-core segment index out of range";
      return false;
    }
    for (int k = 0; k < t.nseg; ++k) {
      const TcSeg& s = tc.segs[t.seg0 + k];
      if (s.kc < 0 || (int64_t)s.ra8 * 8 < t.M || (int64_t)s.rb8 * 8 < t.N || s.pa < 0 ||
          s.pb < 0 || s.pa + (int64_t)s.kc * s.ra8 * kPackTile > nPA ||
          s.pb + (int64_t)s.kc * s.rb8 * kPackTile > nPB) {
        *err = "tensor-core segment out of bounds";
        return false;
      }
      nch[i] += s.kc;
    }
  }
  if (!tc.units.empty()) {
    bool ok = tc.cta_start.size() >= 2 && tc.cta_start.front() == 0 &&
              tc.cta_start.back() == (int32_t)tc.units.size();
    for (size_t i = 1; ok && i < tc.cta_start.size(); ++i) ok = tc.cta_start[i] >= tc.cta_start[i - 1];
    if (!ok) {
      *err = "tensor-core unit schedule";
      return false;
    }
  }
  for (const TcUnit& u : tc.units) {
    if (u.task < 0 || (size_t)u.task >= tasks.size()) {
      *err = "tensor-core unit task out of range";
      return false;
    }
    const GemmTask& t = tasks[u.task];
    if (u.tm < 0 || u.tn < 0 || (int64_t)u.tm * 128 >= t.M || (int64_t)u.tn * 128 >= t.N ||
        u.nchunks != nch[u.task]) {
      *err = "tensor-core unit out of range";
      return false;
    }
  }
  return true;
}

// Tasks whose output is a packed operand (offC = float offset, ldc = R8).
inline bool packed_tasks_ok(const std::vector<GemmTask>& tasks, int64_t nPacked, std::string* err) {
  for (const GemmTask& t : tasks) {
    if (t.M <= 0 || t.N <= 0) continue;
    const int64_t kc = (t.N + 31) / 32;
    if ((int64_t)t.ldc * 8 < t.M || t.offC < 0 || t.offC + kc * t.ldc * kPackTile > nPacked) {
      *err = "packed GEMM output out of bounds";
      return false;
    }
  }
  return true;
}

inline bool packout_ok(const std::vector<CombTask>& tasks, const std::vector<PackOut>& outs,
                       int64_t nPacked, std::string* err) {
  if (outs.size() != tasks.size()) {
    *err = "packed combination table size";
    return false;
  }
  for (size_t i = 0; i < outs.size(); ++i) {
    const PackOut& o = outs[i];
    const int64_t R = o.trans ? tasks[i].cols : tasks[i].rows;
    const int64_t K = o.trans ? tasks[i].rows : tasks[i].cols;
    if ((int64_t)o.R8 * 8 < R || (int64_t)o.KC * 32 < K || o.dst < 0 ||
        o.dst + (int64_t)o.R8 * o.KC * kPackTile > nPacked) {
      *err = "packed combination output out of bounds";
      return false;
    }
  }
  return true;
}

inline bool copies_ok(const std::vector<CopyTask>& tasks, int64_t nSrc, int64_t nDst,
                      int64_t nScale, std::string* err) {
  for (const CopyTask& t : tasks) {
    if (t.rows <= 0 || t.cols <= 0) continue;
    const int64_t ls = t.trans ? (int64_t)(t.cols - 1) * t.ld_s + t.rows - 1
                               : (int64_t)(t.rows - 1) * t.ld_s + t.cols - 1;
    if (!span_ok(t.off_s, ls, nSrc) ||
        !span_ok(t.off_d, (int64_t)(t.rows - 1) * t.ld_d + t.cols - 1, nDst) ||
        (t.rs >= 0 && !span_ok(t.rs, t.rows - 1, nScale)) ||
        (t.cs >= 0 && !span_ok(t.cs, t.cols - 1, nScale))) {
      *err = "block copy out of bounds";
      return false;
    }
  }
  return true;
}

}  // namespace dmrg3s
