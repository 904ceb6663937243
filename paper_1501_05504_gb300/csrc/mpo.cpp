// MPO builders (host): the Hamiltonians of the benchmark workloads as site
// tensors W_i[s_out][s_in][bl][br] (Sec. II: H = W_1 ... W_l).
//
// Layout convention (lower-triangular finite-state form): channel 0 means
// "every term finished", the last channel "nothing placed yet".  The left
// boundary tensor keeps only the last row, the right boundary only column 0.
// A channel's charge is the charge added by the operators already placed.
//
//  XXZ (w = 5): H = J sum_i [(S+_i S-_{i+1} + S-_i S+_{i+1})/2 + Delta Sz_i Sz_{i+1}]
//      channels: 0 done, 1 holds S- (closed by S+), 2 holds S+ (closed by
//      S-), 3 holds Sz, 4 start.  Local basis (up, down), charge 2 S^z.
//  Hubbard (w = 6): H = -t sum_{i,s} (c+_{i,s} c_{i+1,s} + h.c.) + U sum_i n_up n_dn
//      with the Jordan-Wigner string (modes site-major, up before down):
//      c+_i c_{i+1} = (a+ F)_i (a)_{i+1}, c+_{i+1} c_i = (F a)_i (a+)_{i+1}.
//      Local basis index 2 n_up + n_dn, charges (N, 2 S^z).
//  Spin bonds (general two-site couplings, e.g. the snake-ordered cylinder or
//      a ring): channels at each MPO bond: done, then (S+, S-, Sz) held for
//      every site left of the bond with a partner right of it, then start.
//      Spin S = two_s / 2, local basis m = S, S-1, ..., -S, charge 2m, with
//      <m+1|S+|m> = sqrt(S(S+1) - m(m+1)).
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "dmrg3s.h"

namespace {

using Mat = std::vector<double>;   // d x d row-major, [s_out][s_in]

struct SiteT {
  int d = 0, wl = 0, wr = 0, nsym = 0;
  std::vector<double> W;
  std::vector<int32_t> qp, tl, tr;
  void set(int bl, int br, const Mat& op, double coef = 1.0) {
    for (int so = 0; so < d; ++so)
      for (int si = 0; si < d; ++si)
        W[(((size_t)so * d + si) * wl + bl) * wr + br] += coef * op[(size_t)so * d + si];
  }
};

struct Mpo {
  std::vector<SiteT> sites;
};

Mat matmul(const Mat& a, const Mat& b, int d) {
  Mat c((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k)
      for (int j = 0; j < d; ++j) c[(size_t)i * d + j] += a[(size_t)i * d + k] * b[(size_t)k * d + j];
  return c;
}
Mat transpose(const Mat& a, int d) {
  Mat c((size_t)d * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) c[(size_t)j * d + i] = a[(size_t)i * d + j];
  return c;
}
Mat kron2(const Mat& a, const Mat& b) {   // 2x2 (x) 2x2 -> 4x4
  Mat c(16);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) c[(size_t)(2 * i + k) * 4 + (2 * j + l)] = a[i * 2 + j] * b[k * 2 + l];
  return c;
}

// Bulk lower-triangular tensor -> open chain of L sites.
void chain_from_bulk(int L, int d, int w, int nsym, const std::vector<double>& bulk,
                     const std::vector<int32_t>& qp, const std::vector<int32_t>& t, Mpo* out) {
  out->sites.resize(L);
  for (int i = 0; i < L; ++i) {
    SiteT& s = out->sites[i];
    s.d = d;
    s.nsym = nsym;
    const int bl0 = i == 0 ? w - 1 : 0, bl1 = i == 0 ? w : w;
    const int br0 = 0, br1 = i == L - 1 ? 1 : w;
    s.wl = bl1 - bl0;
    s.wr = br1 - br0;
    s.W.assign((size_t)d * d * s.wl * s.wr, 0.0);
    for (int so = 0; so < d; ++so)
      for (int si = 0; si < d; ++si)
        for (int bl = bl0; bl < bl1; ++bl)
          for (int br = br0; br < br1; ++br)
            s.W[(((size_t)so * d + si) * s.wl + (bl - bl0)) * s.wr + (br - br0)] =
                bulk[(((size_t)so * d + si) * w + bl) * w + br];
    s.qp = qp;
    s.tl.assign(t.begin() + (size_t)bl0 * nsym, t.begin() + (size_t)bl1 * nsym);
    s.tr.assign(t.begin() + (size_t)br0 * nsym, t.begin() + (size_t)br1 * nsym);
  }
}

void build_xxz(int L, double J, double Delta, Mpo* out) {
  const int d = 2, w = 5;
  const Mat I = {1, 0, 0, 1}, Sp = {0, 1, 0, 0}, Sm = {0, 0, 1, 0}, Sz = {0.5, 0, 0, -0.5};
  SiteT b;
  b.d = d;
  b.wl = b.wr = w;
  b.W.assign((size_t)d * d * w * w, 0.0);
  b.set(0, 0, I);
  b.set(1, 0, Sp);
  b.set(2, 0, Sm);
  b.set(3, 0, Sz);
  b.set(4, 1, Sm, 0.5 * J);
  b.set(4, 2, Sp, 0.5 * J);
  b.set(4, 3, Sz, J * Delta);
  b.set(4, 4, I);
  chain_from_bulk(L, d, w, 1, b.W, {1, -1}, {0, -2, 2, 0, 0}, out);
}

void build_hubbard(int L, double t, double U, Mpo* out) {
  const int d = 4, w = 6;
  const Mat ann = {0, 1, 0, 0}, par = {1, 0, 0, -1}, I2 = {1, 0, 0, 1};
  const Mat aup = kron2(ann, I2), adn = kron2(par, ann), F = kron2(par, par);
  Mat I4(16, 0.0);
  for (int k = 0; k < 4; ++k) I4[k * 5] = 1.0;
  const Mat nup = matmul(transpose(aup, d), aup, d), ndn = matmul(transpose(adn, d), adn, d);
  SiteT b;
  b.d = d;
  b.wl = b.wr = w;
  b.W.assign((size_t)d * d * w * w, 0.0);
  b.set(0, 0, I4);
  b.set(1, 0, aup);
  b.set(2, 0, transpose(aup, d));
  b.set(3, 0, adn);
  b.set(4, 0, transpose(adn, d));
  b.set(5, 0, matmul(nup, ndn, d), U);
  b.set(5, 1, matmul(transpose(aup, d), F, d), -t);
  b.set(5, 2, matmul(F, aup, d), -t);
  b.set(5, 3, matmul(transpose(adn, d), F, d), -t);
  b.set(5, 4, matmul(F, adn, d), -t);
  b.set(5, 5, I4);
  chain_from_bulk(L, d, w, 2, b.W, {0, 0, 1, -1, 1, 1, 2, 0},
                  {0, 0, 1, 1, -1, -1, 1, -1, -1, 1, 0, 0}, out);
}

// bonds: nb entries (i, j) with i < j, couplings (Jxy, Jz); spin two_s / 2
dmrg3s_status build_spin_bonds(int L, int nb, const int32_t* ij, const double* J, int two_s,
                               Mpo* out) {
  const int d = two_s + 1;
  const double S = 0.5 * two_s;
  Mat I((size_t)d * d, 0.0), Sp((size_t)d * d, 0.0), Sz((size_t)d * d, 0.0);
  std::vector<int32_t> qp(d);
  for (int k = 0; k < d; ++k) {
    const double m = S - k;
    I[(size_t)k * d + k] = 1.0;
    Sz[(size_t)k * d + k] = m;
    qp[k] = two_s - 2 * k;
    if (k > 0) Sp[(size_t)(k - 1) * d + k] = std::sqrt(S * (S + 1.0) - m * (m + 1.0));
  }
  const Mat Sm = transpose(Sp, d);
  std::map<int, std::vector<std::pair<int, std::pair<double, double>>>> partners;
  for (int k = 0; k < nb; ++k) {
    const int i = ij[2 * k], j = ij[2 * k + 1];
    if (!(0 <= i && i < j && j < L)) return DMRG3S_ERR_ARG;
    partners[i].push_back({j, {J[2 * k], J[2 * k + 1]}});
  }
  // channels at MPO bond k (left of site k): done, (s, op) for open sites, start
  struct Ch {
    int kind, site, op;   // kind 0 done, 1 open, 2 start; op 0 S+, 1 S-, 2 Sz
  };
  std::vector<std::vector<Ch>> chans(L + 1);
  for (int k = 0; k <= L; ++k) {
    std::set<int> open;
    for (int q = 0; q < nb; ++q)
      if (ij[2 * q] < k && k <= ij[2 * q + 1]) open.insert(ij[2 * q]);
    if (k == 0) {
      chans[k] = {{2, -1, -1}};
    } else if (k == L) {
      chans[k] = {{0, -1, -1}};
    } else {
      chans[k].push_back({0, -1, -1});
      for (int s : open)
        for (int op = 0; op < 3; ++op) chans[k].push_back({1, s, op});
      chans[k].push_back({2, -1, -1});
    }
  }
  auto index = [&](int k, int kind, int site, int op) {
    for (size_t n = 0; n < chans[k].size(); ++n) {
      const Ch& c = chans[k][n];
      if (c.kind == kind && (kind != 1 || (c.site == site && c.op == op))) return (int)n;
    }
    return -1;
  };
  const Mat ops[3] = {Sp, Sm, Sz};
  const int charge[3] = {2, -2, 0};
  out->sites.resize(L);
  for (int i = 0; i < L; ++i) {
    SiteT& s = out->sites[i];
    s.d = d;
    s.nsym = 1;
    s.wl = (int)chans[i].size();
    s.wr = (int)chans[i + 1].size();
    s.W.assign((size_t)d * d * s.wl * s.wr, 0.0);
    s.qp = qp;
    for (const Ch& c : chans[i]) s.tl.push_back(c.kind == 1 ? charge[c.op] : 0);
    for (const Ch& c : chans[i + 1]) s.tr.push_back(c.kind == 1 ? charge[c.op] : 0);
    const int dl = index(i, 0, 0, 0), dr = index(i + 1, 0, 0, 0);
    const int sl = index(i, 2, 0, 0), sr = index(i + 1, 2, 0, 0);
    if (dl >= 0 && dr >= 0) s.set(dl, dr, I);
    if (sl >= 0 && sr >= 0) s.set(sl, sr, I);
    if (sl >= 0)
      for (int op = 0; op < 3; ++op) {
        const int r = index(i + 1, 1, i, op);
        if (r >= 0) s.set(sl, r, ops[op]);
      }
    for (size_t n = 0; n < chans[i].size(); ++n) {
      const Ch& c = chans[i][n];
      if (c.kind != 1) continue;
      const int r = index(i + 1, 1, c.site, c.op);
      if (r >= 0) s.set((int)n, r, I);
      for (auto& pj : partners[c.site]) {
        if (pj.first != i) continue;
        // S+ is closed by S- (Jxy/2), S- by S+ (Jxy/2), Sz by Sz (Jz)
        if (c.op == 0) s.set((int)n, dr, Sm, 0.5 * pj.second.first);
        if (c.op == 1) s.set((int)n, dr, Sp, 0.5 * pj.second.first);
        if (c.op == 2) s.set((int)n, dr, Sz, pj.second.second);
      }
    }
  }
  return DMRG3S_OK;
}

}  // namespace

struct dmrg3s_mpo_s {
  Mpo m;
};

extern "C" {

dmrg3s_status dmrg3s_mpo_create(int32_t model, int32_t nsites, const double* params,
                                int32_t nbonds, const int32_t* bonds, const double* couplings,
                                dmrg3s_mpo* out) {
  if (!out || nsites < 2) return DMRG3S_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<dmrg3s_mpo_s> h(new dmrg3s_mpo_s());
  switch (model) {
    case DMRG3S_MODEL_XXZ:
      if (!params) return DMRG3S_ERR_ARG;
      build_xxz(nsites, params[0], params[1], &h->m);
      break;
    case DMRG3S_MODEL_HUBBARD:
      if (!params) return DMRG3S_ERR_ARG;
      build_hubbard(nsites, params[0], params[1], &h->m);
      break;
    case DMRG3S_MODEL_SPIN_BONDS: {
      if (nbonds < 1 || !bonds || !couplings) return DMRG3S_ERR_ARG;
      int two_s = 1;
      if (params) {
        if (!(params[0] >= 1.0 && params[0] <= 8.0) || params[0] != (double)(int)params[0])
          return DMRG3S_ERR_ARG;
        two_s = (int)params[0];
      }
      dmrg3s_status s = build_spin_bonds(nsites, nbonds, bonds, couplings, two_s, &h->m);
      if (s != DMRG3S_OK) return s;
      break;
    }
    default:
      return DMRG3S_ERR_ARG;
  }
  *out = h.release();
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_mpo_destroy(dmrg3s_mpo mpo) {
  if (!mpo) return DMRG3S_ERR_ARG;
  delete mpo;
  return DMRG3S_OK;
}

dmrg3s_status dmrg3s_mpo_get_site(dmrg3s_mpo mpo, int32_t i, dmrg3s_mpo_site* site) {
  if (!mpo || !site || i < 0 || i >= (int)mpo->m.sites.size()) return DMRG3S_ERR_ARG;
  const SiteT& s = mpo->m.sites[i];
  site->nsym = s.nsym;
  site->d = s.d;
  site->wl = s.wl;
  site->wr = s.wr;
  site->qp = s.qp.data();
  site->tl = s.tl.data();
  site->tr = s.tr.data();
  site->W = s.W.data();
  return DMRG3S_OK;
}

}  // extern "C"
