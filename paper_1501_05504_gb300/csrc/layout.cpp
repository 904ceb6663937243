// Block-sparse layouts (host side).  See layout.hpp.
#include "layout.hpp"

#include <algorithm>
#include <map>

namespace dmrg3s {

int Bond::find(const Charge& c) const {
  if (nsym == 0) return 0;
  auto it = std::lower_bound(q.begin(), q.end(), c);
  if (it != q.end() && *it == c) return (int)(it - q.begin());
  return -1;
}

static dmrg3s_status read_charges(int nsym, int n, const int32_t* src, std::vector<Charge>* out,
                                  std::string* err, const char* what) {
  out->assign(n, Charge{});
  if (nsym == 0) return DMRG3S_OK;
  if (!src) {
    *err = std::string(what) + ": charge table is NULL";
    return DMRG3S_ERR_ARG;
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < nsym; ++k) (*out)[i][k] = src[(size_t)i * nsym + k];
  return DMRG3S_OK;
}

dmrg3s_status make_bond(int nsym, const dmrg3s_bond* b, Bond* out, std::string* err) {
  if (nsym < 0 || nsym > kMaxSym) {
    *err = "nsym must be 0, 1 or 2";
    return DMRG3S_ERR_ARG;
  }
  if (!b || b->nsec < 1 || !b->dim) {
    *err = "bond: nsec must be >= 1 with a dim table";
    return DMRG3S_ERR_ARG;
  }
  if (nsym == 0 && b->nsec != 1) {
    *err = "bond: a bond without symmetry has exactly one sector";
    return DMRG3S_ERR_QN;
  }
  out->nsym = nsym;
  dmrg3s_status st = read_charges(nsym, b->nsec, b->q, &out->q, err, "bond");
  if (st != DMRG3S_OK) return st;
  out->dim.assign(b->dim, b->dim + b->nsec);
  out->off.assign(b->nsec + 1, 0);
  for (int i = 0; i < b->nsec; ++i) {
    if (out->dim[i] < 1) {
      *err = "bond: sector dimensions must be >= 1";
      return DMRG3S_ERR_ARG;
    }
    if (i > 0 && !(out->q[i - 1] < out->q[i])) {
      *err = "bond: sector charges must be strictly increasing";
      return DMRG3S_ERR_QN;
    }
    out->off[i + 1] = out->off[i] + out->dim[i];
  }
  out->total = out->off[b->nsec];
  return DMRG3S_OK;
}

dmrg3s_status make_site_from(int nsym, int d, const std::vector<Charge>& qp, const Bond& left,
                             const Bond& right, SiteLayout* out) {
  out->nsym = nsym;
  out->d = d;
  out->qp = qp;
  out->left = left;
  out->right = right;
  out->blocks.clear();
  out->index.assign((size_t)d * left.nsec(), -1);
  int64_t off = 0;
  for (int s = 0; s < d; ++s)
    for (int i = 0; i < left.nsec(); ++i) {
      int j = right.find(add(left.q[i], qp[s]));
      if (j < 0) continue;
      out->index[(size_t)s * left.nsec() + i] = (int)out->blocks.size();
      out->blocks.push_back(Block{s, i, j, off, left.dim[i], right.dim[j]});
      off += left.dim[i] * right.dim[j];
    }
  out->size = off;
  return DMRG3S_OK;
}

dmrg3s_status make_site(const dmrg3s_site* s, SiteLayout* out, std::string* err) {
  if (!s) {
    *err = "site tensor is NULL";
    return DMRG3S_ERR_ARG;
  }
  if (s->d < 1) {
    *err = "site tensor: d must be >= 1";
    return DMRG3S_ERR_ARG;
  }
  Bond l, r;
  dmrg3s_status st = make_bond(s->nsym, &s->left, &l, err);
  if (st != DMRG3S_OK) return st;
  st = make_bond(s->nsym, &s->right, &r, err);
  if (st != DMRG3S_OK) return st;
  std::vector<Charge> qp;
  st = read_charges(s->nsym, s->d, s->qp, &qp, err, "site qp");
  if (st != DMRG3S_OK) return st;
  return make_site_from(s->nsym, s->d, qp, l, r, out);
}

dmrg3s_status make_env_from(int nsym, int w, const std::vector<Charge>& t, const Bond& bond,
                            EnvLayout* out) {
  out->nsym = nsym;
  out->w = w;
  out->t = t;
  out->bond = bond;
  out->blocks.clear();
  out->index.assign((size_t)w * bond.nsec(), -1);
  int64_t off = 0;
  for (int b = 0; b < w; ++b)
    for (int ik = 0; ik < bond.nsec(); ++ik) {
      int ib = bond.find(add(bond.q[ik], t[b]));
      if (ib < 0) continue;
      out->index[(size_t)b * bond.nsec() + ik] = (int)out->blocks.size();
      out->blocks.push_back(Block{b, ib, ik, off, bond.dim[ib], bond.dim[ik]});
      off += bond.dim[ib] * bond.dim[ik];
    }
  out->size = off;
  return DMRG3S_OK;
}

dmrg3s_status make_env(const dmrg3s_env* e, EnvLayout* out, std::string* err) {
  if (!e) {
    *err = "environment is NULL";
    return DMRG3S_ERR_ARG;
  }
  if (e->w < 1) {
    *err = "environment: w must be >= 1";
    return DMRG3S_ERR_ARG;
  }
  Bond b;
  dmrg3s_status st = make_bond(e->nsym, &e->bond, &b, err);
  if (st != DMRG3S_OK) return st;
  std::vector<Charge> t;
  st = read_charges(e->nsym, e->w, e->t, &t, err, "environment t");
  if (st != DMRG3S_OK) return st;
  return make_env_from(e->nsym, e->w, t, b, out);
}

dmrg3s_status make_mpo(const dmrg3s_mpo_site* w, MpoLayout* out, std::string* err) {
  if (!w || !w->W) {
    *err = "MPO site or its W table is NULL";
    return DMRG3S_ERR_ARG;
  }
  if (w->nsym < 0 || w->nsym > kMaxSym || w->d < 1 || w->wl < 1 || w->wr < 1) {
    *err = "MPO site: bad nsym/d/wl/wr";
    return DMRG3S_ERR_ARG;
  }
  out->nsym = w->nsym;
  out->d = w->d;
  out->wl = w->wl;
  out->wr = w->wr;
  dmrg3s_status st = read_charges(w->nsym, w->d, w->qp, &out->qp, err, "MPO qp");
  if (st != DMRG3S_OK) return st;
  st = read_charges(w->nsym, w->wl, w->tl, &out->tl, err, "MPO tl");
  if (st != DMRG3S_OK) return st;
  st = read_charges(w->nsym, w->wr, w->tr, &out->tr, err, "MPO tr");
  if (st != DMRG3S_OK) return st;
  size_t n = (size_t)w->d * w->d * w->wl * w->wr;
  out->W.assign(w->W, w->W + n);
  for (int so = 0; so < w->d; ++so)
    for (int si = 0; si < w->d; ++si)
      for (int bl = 0; bl < w->wl; ++bl)
        for (int br = 0; br < w->wr; ++br) {
          double v = out->at(so, si, bl, br);
          if (v == 0.0) continue;
          if (v != v) {
            *err = "MPO site: NaN entry";
            return DMRG3S_ERR_NUMERIC;
          }
          Charge lhs = add(sub(out->qp[so], out->qp[si]), out->tl[bl]);
          if (!(lhs == out->tr[br])) {
            *err = "MPO site: non-zero entry breaks charge conservation";
            return DMRG3S_ERR_QN;
          }
        }
  return DMRG3S_OK;
}

dmrg3s_status fuse_bond(const Bond& src, int w, const std::vector<Charge>& t, bool include_base,
                        FusedBond* out) {
  std::map<Charge, int64_t> size;
  if (src.nsym == 0) {
    // without symmetry everything lands in the single sector
    Bond b;
    b.nsym = 0;
    b.q.assign(1, Charge{});
    int64_t tot = include_base ? src.total : 0;
    out->target.assign((size_t)w * src.nsec(), 0);
    out->offset.assign((size_t)w * src.nsec(), 0);
    out->base_target.assign(src.nsec(), include_base ? 0 : -1);
    for (int bb = 0; bb < w; ++bb) {
      out->offset[bb] = tot;
      tot += src.total;
    }
    b.dim.assign(1, tot);
    b.off = {0, tot};
    b.total = tot;
    out->bond = b;
    return DMRG3S_OK;
  }
  if (include_base)
    for (int j = 0; j < src.nsec(); ++j) size[src.q[j]] += src.dim[j];
  for (int bb = 0; bb < w; ++bb)
    for (int j = 0; j < src.nsec(); ++j) size[add(src.q[j], t[bb])] += src.dim[j];
  Bond b;
  b.nsym = src.nsym;
  for (auto& kv : size) {
    b.q.push_back(kv.first);
    b.dim.push_back(kv.second);
  }
  b.off.assign(b.dim.size() + 1, 0);
  for (size_t k = 0; k < b.dim.size(); ++k) b.off[k + 1] = b.off[k] + b.dim[k];
  b.total = b.off.back();
  std::vector<int64_t> fill(b.dim.size(), 0);
  out->base_target.assign(src.nsec(), -1);
  if (include_base)
    for (int j = 0; j < src.nsec(); ++j) {
      int k = b.find(src.q[j]);
      out->base_target[j] = k;
      fill[k] += src.dim[j];
    }
  out->target.assign((size_t)w * src.nsec(), -1);
  out->offset.assign((size_t)w * src.nsec(), 0);
  for (int bb = 0; bb < w; ++bb)
    for (int j = 0; j < src.nsec(); ++j) {
      int k = b.find(add(src.q[j], t[bb]));
      out->target[(size_t)bb * src.nsec() + j] = k;
      out->offset[(size_t)bb * src.nsec() + j] = fill[k];
      fill[k] += src.dim[j];
    }
  out->bond = b;
  return DMRG3S_OK;
}

bool same_bond(const Bond& a, const Bond& b) {
  if (a.nsym != b.nsym || a.dim != b.dim) return false;
  if (a.nsym == 0) return true;
  return a.q == b.q;
}

bool same_charges(const std::vector<Charge>& a, const std::vector<Charge>& b) { return a == b; }

}  // namespace dmrg3s
