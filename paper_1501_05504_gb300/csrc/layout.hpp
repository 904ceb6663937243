// Block-sparse layouts of MPS site tensors and environments (host side).
//
// A bond is a list of charge sectors.  The selection rules are those of
// charge conservation for the tensors of Sec. II of arXiv:1501.05504:
//   site tensor  M[s](al, ar):   q_right[j] == q_left[i] + qp[s]
//   environment  E[b](a', a):    q[ib]      == q[ik] + t[b]
//   MPO tensor   W[s',s,bl,br]:  qp[s'] - qp[s] + tl[bl] == tr[br]
// Blocks are stored row-major and packed in the canonical order documented in
// include/dmrg3s.h.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "dmrg3s.h"

namespace dmrg3s {

constexpr int kMaxSym = DMRG3S_MAX_NSYM;
using Charge = std::array<int32_t, kMaxSym>;

inline Charge add(const Charge& a, const Charge& b) {
  Charge c{};
  for (int k = 0; k < kMaxSym; ++k) c[k] = a[k] + b[k];
  return c;
}
inline Charge sub(const Charge& a, const Charge& b) {
  Charge c{};
  for (int k = 0; k < kMaxSym; ++k) c[k] = a[k] - b[k];
  return c;
}

struct Bond {
  int nsym = 0;
  std::vector<Charge> q;
  std::vector<int64_t> dim;
  std::vector<int64_t> off;   // prefix sums of dim (dense position of a sector)
  int64_t total = 0;
  int nsec() const { return (int)dim.size(); }
  int find(const Charge& c) const;   // sector index with charge c, or -1
};

struct Block {
  int a, b, c;        // (s, i, j) for sites; (b, ib, ik) for environments
  int64_t off;        // element offset of the block
  int64_t rows, cols;
};

struct SiteLayout {
  int nsym = 0, d = 0;
  std::vector<Charge> qp;
  Bond left, right;
  std::vector<Block> blocks;              // canonical order
  std::vector<int> index;                 // [s * nsec_left + i] -> block or -1
  int64_t size = 0;
  int block_of(int s, int i) const { return index[(size_t)s * left.nsec() + i]; }
};

struct EnvLayout {
  int nsym = 0, w = 0;
  std::vector<Charge> t;
  Bond bond;
  std::vector<Block> blocks;
  std::vector<int> index;                 // [b * nsec + ik] -> block or -1
  int64_t size = 0;
  int block_of(int b, int ik) const { return index[(size_t)b * bond.nsec() + ik]; }
};

struct MpoLayout {
  int nsym = 0, d = 0, wl = 0, wr = 0;
  std::vector<Charge> qp, tl, tr;
  std::vector<double> W;                  // [s'][s][bl][br]
  double at(int so, int si, int bl, int br) const {
    return W[(((size_t)so * d + si) * wl + bl) * wr + br];
  }
};

// Each returns DMRG3S_OK or an error status with a message in *err.
dmrg3s_status make_bond(int nsym, const dmrg3s_bond* b, Bond* out, std::string* err);
dmrg3s_status make_site(const dmrg3s_site* s, SiteLayout* out, std::string* err);
dmrg3s_status make_env(const dmrg3s_env* e, EnvLayout* out, std::string* err);
dmrg3s_status make_mpo(const dmrg3s_mpo_site* w, MpoLayout* out, std::string* err);
dmrg3s_status make_site_from(int nsym, int d, const std::vector<Charge>& qp, const Bond& left,
                             const Bond& right, SiteLayout* out);
dmrg3s_status make_env_from(int nsym, int w, const std::vector<Charge>& t, const Bond& bond,
                            EnvLayout* out);

// Fused bond of the expansion (Sec. IV A): sectors q + t[b].
struct FusedBond {
  Bond bond;                                 // the fused bond
  // for every (channel b, source sector j): target sector and row/column offset
  // of the D_j states inside that sector (after the base part when included)
  std::vector<int> target;                   // [b * nsec_src + j] -> fused sector or -1
  std::vector<int64_t> offset;               // [b * nsec_src + j] -> offset inside sector
  std::vector<int> base_target;              // [j] -> fused sector of the base states
};
dmrg3s_status fuse_bond(const Bond& src, int w, const std::vector<Charge>& t, bool include_base,
                        FusedBond* out);

bool same_bond(const Bond& a, const Bond& b);
bool same_charges(const std::vector<Charge>& a, const std::vector<Charge>& b);

}  // namespace dmrg3s
