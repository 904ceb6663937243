// Host-side bounds validation of task tables before any launch: every element
// a kernel will read or write must lie inside the buffer it addresses.  A
// violation is an internal planning error and is reported as a status, so a
// bad table never reaches the device.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kernels.hpp"
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
