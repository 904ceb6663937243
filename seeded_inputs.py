"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and the benchmark.

This module holds none of the method's arithmetic: it only draws random
numbers into block structures (which blocks exist follows from charge
conservation, i.e. from the sparsity pattern alone).  Both implementations
receive the same arrays and each does its own packing.

Neutral representation
----------------------
* a *bond* is ``{"q": int64 (nsec, nsym), "dim": int64 (nsec,)}`` with the
  sectors in lexicographic charge order;
* a *site tensor* ``M[s](al, ar)`` is ``{"qp": (d, nsym), "left": bond,
  "right": bond, "blocks": {(s, i, j): float64 (D_l[i], D_r[j])}}`` with a
  block wherever ``q_l[i] + qp[s] == q_r[j]``;
* an *environment* ``E[b](a_bra, a_ket)`` is ``{"t": (w, nsym), "bra": bond,
  "ket": bond, "blocks": {(b, i_bra, i_ket): (D[i_bra], D[i_ket])}}`` with a
  block wherever ``q_ket[i_ket] + t[b] == q_bra[i_bra]``;
* an *MPO site* is ``{"qp", "tl", "tr", "W": float64 (d, d, wl, wr)}`` indexed
  ``W[s_out, s_in, bl, br]``.

Workload shapes (synthetic stand-ins for converged DMRG states)
-----------------------------------------------------------------
Sector dimensions follow a discretised Gaussian in the charges around the
mean charge of the bond, normalised to the requested bond dimension ``m``
(every sector at least one state).  The widths are chosen to resemble the
Schmidt-spectrum distributions of the paper's one-dimensional workloads (a
few dominant S^z sectors, tails of size one).
"""
import itertools

import numpy as np

SEED_BASE = 1000


def rng_for(tag):
    """Deterministic generator for a named workload (``1000 + config number`` style seeds)."""
    if isinstance(tag, (int, np.integer)):
        return np.random.default_rng(int(tag))
    h = 0
    for ch in str(tag):
        h = (h * 131 + ord(ch)) % (2 ** 31)
    return np.random.default_rng(h)


# ---- bonds ---------------------------------------------------------------------

def bond(q, dim):
    q = np.asarray(q, dtype=np.int64)
    if q.ndim == 1:
        q = q.reshape(-1, 1)
    dim = np.asarray(dim, dtype=np.int64)
    order = sorted(range(len(dim)), key=lambda n: tuple(q[n]))
    return {"q": q[order].copy(), "dim": dim[order].copy()}


def dense_bond(m):
    return {"q": np.zeros((1, 0), dtype=np.int64), "dim": np.array([m], dtype=np.int64)}


def gaussian_bond(m, centre, sigma, step, span):
    """Sectors on a charge grid around ``centre`` with Gaussian weights, total dim m.

    ``centre``, ``sigma``, ``step`` and ``span`` are per-charge tuples; the grid
    runs over centre + step*k for |k| <= span.
    """
    centre = np.atleast_1d(centre)
    sigma = np.atleast_1d(sigma).astype(float)
    step = np.atleast_1d(step)
    span = np.atleast_1d(span)
    axes = [centre[k] + step[k] * np.arange(-span[k], span[k] + 1) for k in range(len(centre))]
    qs = np.array(list(itertools.product(*axes)), dtype=np.int64)
    wts = np.exp(-np.sum(((qs - centre[None, :]) / sigma[None, :]) ** 2, axis=1) / 2.0)
    raw = wts / wts.sum() * m
    dims = np.maximum(1, np.floor(raw)).astype(np.int64)
    # distribute the remainder to the largest fractional parts, then trim from the largest
    while dims.sum() < m:
        n = int(np.argmax(raw - dims))
        dims[n] += 1
    while dims.sum() > m:
        n = int(np.argmax(dims))
        dims[n] -= 1
    keep = dims > 0
    return bond(qs[keep], dims[keep])


# ---- structure enumeration ---------------------------------------------------------

def _find(bnd, qvec):
    hit = np.nonzero(np.all(bnd["q"] == np.asarray(qvec)[None, :], axis=1))[0]
    return int(hit[0]) if len(hit) else -1


def site_block_keys(qp, left, right):
    keys = []
    for s in range(qp.shape[0]):
        for i in range(len(left["dim"])):
            j = _find(right, left["q"][i] + qp[s]) if qp.shape[1] else 0
            if j >= 0:
                keys.append((s, i, j))
    return keys


def env_block_keys(t, bra, ket):
    keys = []
    for b in range(t.shape[0]):
        for i in range(len(ket["dim"])):
            ib = _find(bra, ket["q"][i] + t[b]) if t.shape[1] else 0
            if ib >= 0:
                keys.append((b, ib, i))
    return keys


# ---- random tensors ---------------------------------------------------------------

def random_site(rng, qp, left, right, scale=1.0):
    blocks = {}
    for (s, i, j) in site_block_keys(qp, left, right):
        blocks[(s, i, j)] = scale * rng.standard_normal((int(left["dim"][i]), int(right["dim"][j])))
    return {"qp": np.asarray(qp, dtype=np.int64), "left": left, "right": right, "blocks": blocks}


def random_env(rng, t, bra, ket, scale=None):
    blocks = {}
    for (b, ib, ik) in env_block_keys(t, bra, ket):
        db, dk = int(bra["dim"][ib]), int(ket["dim"][ik])
        sc = scale if scale is not None else 1.0 / np.sqrt(max(dk, 1))
        blocks[(b, ib, ik)] = sc * rng.standard_normal((db, dk))
    return {"t": np.asarray(t, dtype=np.int64), "bra": bra, "ket": ket, "blocks": blocks}


def random_mpo_site(rng, qp, tl, tr, density=1.0):
    """Random W[s_out, s_in, bl, br] on the charge-allowed entries (a fraction ``density`` kept)."""
    qp, tl, tr = (np.asarray(x, dtype=np.int64) for x in (qp, tl, tr))
    d, wl, wr = qp.shape[0], tl.shape[0], tr.shape[0]
    W = np.zeros((d, d, wl, wr))
    for so, si, bl, br in itertools.product(range(d), range(d), range(wl), range(wr)):
        ok = True if qp.shape[1] == 0 else np.all(qp[so] - qp[si] + tl[bl] == tr[br])
        if ok and rng.random() < density:
            W[so, si, bl, br] = rng.standard_normal()
    return {"qp": qp, "tl": tl, "tr": tr, "W": W}


def symmetric_mpo_site(rng, qp, tl, tr, density=1.0):
    """Random W with W[s, s', b_bar, c_bar] = W[s', s, b, c] (a symmetric H_eff).

    Left and right channels are paired by charge negation (``conjugate_channels``).
    """
    W = random_mpo_site(rng, qp, tl, tr, density)
    pl, pr = conjugate_channels(np.asarray(tl)), conjugate_channels(np.asarray(tr))
    A = W["W"]
    B = np.transpose(A, (1, 0, 2, 3))[:, :, pl, :][:, :, :, pr]
    W["W"] = 0.5 * (A + B)
    return W


def conjugate_channels(t):
    """Pairing b -> b_bar with t[b_bar] = -t[b] (first match, self-paired when t == 0)."""
    w = t.shape[0]
    pair = -np.ones(w, dtype=np.int64)
    for b in range(w):
        if pair[b] >= 0:
            continue
        if t.shape[1] == 0 or np.all(t[b] == 0):
            pair[b] = b
            continue
        for c in range(w):
            if pair[c] < 0 and c != b and np.all(t[c] == -t[b]):
                pair[b], pair[c] = c, b
                break
        if pair[b] < 0:
            raise ValueError("channel charges are not closed under negation")
    return pair


def symmetric_env(rng, t, bnd, identity_channels=(), scale=None):
    """Environment E[b] with E[b_bar] = E[b]^T (so that H_eff is symmetric).

    Channels listed in ``identity_channels`` hold the identity matrix, as the
    "nothing placed yet" channel of a left-normalised left environment does.
    """
    t = np.asarray(t, dtype=np.int64)
    pair = conjugate_channels(t)
    e = random_env(rng, t, bnd, bnd, scale=scale)
    blk = e["blocks"]
    for (b, ib, ik) in list(blk.keys()):
        bb = int(pair[b])
        if b in identity_channels:
            blk[(b, ib, ik)] = np.eye(blk[(b, ib, ik)].shape[0]) if ib == ik else 0.0 * blk[(b, ib, ik)]
        elif bb == b:
            if ib == ik:
                X = blk[(b, ib, ik)]
                blk[(b, ib, ik)] = 0.5 * (X + X.T)
            elif (b, ik, ib) in blk and ib > ik:
                blk[(b, ib, ik)] = blk[(b, ik, ib)].T.copy()
        elif bb < b:
            blk[(b, ib, ik)] = blk[(bb, ik, ib)].T.copy()
    return e


# ---- MPS initial states -------------------------------------------------------------

def random_dense_mps(rng, L, d, m_max):
    """N(0,1) site tensors with bond dims min(d^i, d^(l-i), m_max) (not normalised)."""
    dims = [min(d ** i, d ** (L - i), m_max) for i in range(L + 1)]
    return [rng.standard_normal((d, dims[i], dims[i + 1])) for i in range(L)]


def product_state_sites(qp, local_states):
    """Neutral site tensors (m = 1) of a product state |s_1 ... s_l>.

    The bond charges accumulate the local charges from the left, as the
    selection rule of a site tensor requires.
    """
    qp = np.asarray(qp, dtype=np.int64)
    nsym = qp.shape[1]
    q = np.zeros(nsym, dtype=np.int64)
    sites = []
    for s in local_states:
        left = {"q": q.reshape(1, nsym).copy(), "dim": np.array([1], dtype=np.int64)}
        q = q + qp[s]
        right = {"q": q.reshape(1, nsym).copy(), "dim": np.array([1], dtype=np.int64)}
        sites.append({"qp": qp, "left": left, "right": right, "blocks": {(int(s), 0, 0): np.ones((1, 1))}})
    return sites


def dense_mps_sites(tensors):
    """Neutral site tensors (no symmetry) of dense arrays M[s, al, ar]."""
    out = []
    for T in tensors:
        d, ml, mr = T.shape
        out.append({"qp": np.zeros((d, 0), dtype=np.int64), "left": dense_bond(ml),
                    "right": dense_bond(mr),
                    "blocks": {(s, 0, 0): np.array(T[s]) for s in range(d)}})
    return out


# ---- named workloads ---------------------------------------------------------------

XXZ_QP = np.array([[1], [-1]], dtype=np.int64)
XXZ_T = np.array([[0], [-2], [2], [0], [0]], dtype=np.int64)
HUB_QP = np.array([[0, 0], [1, -1], [1, 1], [2, 0]], dtype=np.int64)
HUB_T = np.array([[0, 0], [1, 1], [-1, -1], [1, -1], [-1, 1], [0, 0]], dtype=np.int64)

WORKLOADS = {
    # name: (description, d, w, m, charge model)
    "heisenberg_l20_m64_dense": "S=1/2 Heisenberg chain, L=20, d=2, w=5, m_max=64, no symmetry blocks",
    "xxz_l100_m512_u1": "XXZ chain Delta=1, L=100, d=2, w=5, U(1) S^z blocks, m_max=512 (central site)",
    "hubbard_l64_m1024_u1u1": "Fermi-Hubbard L=64, d=4, w=6, U(1)xU(1) (N, S^z) blocks, m_max=1024 (central site)",
    "cylinder_4x16_m2048_u1": "J1 Heisenberg 4x16 cylinder, d=2, w=14, U(1) S^z blocks, m_max=2048 (central site)",
}


def central_bonds(name, m=None):
    """(left bond, right bond) of the central site of a named workload."""
    if name == "xxz_l100_m512_u1":
        m = m or 512
        left = gaussian_bond(m, centre=(1,), sigma=(3.0,), step=(2,), span=(6,))
        right = gaussian_bond(m, centre=(0,), sigma=(3.0,), step=(2,), span=(6,))
        return left, right
    if name == "hubbard_l64_m1024_u1u1":
        m = m or 1024
        left = gaussian_bond(m, centre=(31, 1), sigma=(2.0, 2.0), step=(1, 2), span=(5, 4))
        right = gaussian_bond(m, centre=(32, 0), sigma=(2.0, 2.0), step=(1, 2), span=(5, 4))
        # only charge combinations with matching parity (N + 2Sz even) exist for fermions
        return _parity_filter(left, m), _parity_filter(right, m)
    if name == "cylinder_4x16_m2048_u1":
        m = m or 2048
        left = gaussian_bond(m, centre=(1,), sigma=(5.0,), step=(2,), span=(8,))
        right = gaussian_bond(m, centre=(0,), sigma=(5.0,), step=(2,), span=(8,))
        return left, right
    if name == "heisenberg_l20_m64_dense":
        m = m or 64
        return dense_bond(m), dense_bond(m)
    raise KeyError(name)


def _parity_filter(bnd, m):
    q = bnd["q"]
    ok = (q[:, 0] + q[:, 1]) % 2 == 0
    q2, d2 = q[ok], bnd["dim"][ok].astype(float)
    d2 = np.maximum(1, np.round(d2 / d2.sum() * m)).astype(np.int64)
    while d2.sum() > m:
        d2[int(np.argmax(d2))] -= 1
    while d2.sum() < m:
        d2[int(np.argmax(d2))] += 1
    return bond(q2, d2)


# ---- batched chains --------------------------------------------------------------

BATCH_M_CHOICES = (64, 128, 256, 512)


def batch_xxz_chains(n=64, seed=1005):
    """The batched-chain workload: n independent open XXZ chains, J = 1, with
    L drawn uniformly from the even lengths 16, 18, ..., 128 (an S^z = 0
    sector needs an even length), Delta uniformly from [0.5, 1.5] and m_max
    uniformly from BATCH_M_CHOICES, in that order per chain, from
    numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = 2 * int(rng.integers(8, 65))
        delta = float(rng.uniform(0.5, 1.5))
        m = int(BATCH_M_CHOICES[int(rng.integers(0, len(BATCH_M_CHOICES)))])
        out.append({"L": L, "J": 1.0, "Delta": delta, "m_max": m})
    return out
