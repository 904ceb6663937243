"""Test-side helpers for GPU-vs-oracle parity: problem generation and layout mapping.

Inputs come from ``seeded_inputs``; the oracle gets dense arrays through
``oracle.io``, the CUDA path gets canonical flat buffers through the binding.
This module only moves numbers between the two layouts.
"""
import numpy as np

import seeded_inputs as si
from oracle import io

FP64_TOL = 1e-12        # relative Frobenius error, FP64 path vs FP64 oracle
TF32X3_TOL = 1e-6       # relative Frobenius error of 3xTF32 with FP32 accumulation
# Per-block max-relative bounds (block_rel_err): one element of a block against
# the block's largest entry, so a factor ~10 above the Frobenius bounds.
FP64_BLOCK_TOL = 1e-11
TF32X3_BLOCK_TOL = 1e-5


def rel_err(got, ref):
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def block_rel_err(got, ref, parts):
    """Largest per-block relative error max|got - ref| / max|ref| over the charge
    blocks of a dense array, so that a wrong small sector cannot hide under the
    Frobenius norm of the large ones.

    parts: one sequence of sector dimensions per axis (an axis without sectors,
    such as the physical index or the MPO channel, is given as [1] * size).
    A block whose reference is zero must be zero in ``got`` too, up to 1e-300
    of nothing: its error is taken relative to the largest reference entry.
    """
    offs = [np.concatenate([[0], np.cumsum(np.asarray(p, dtype=np.int64))]) for p in parts]
    assert tuple(int(o[-1]) for o in offs) == ref.shape == got.shape
    gmax = float(np.abs(ref).max()) if ref.size else 0.0
    worst = 0.0
    for idx in np.ndindex(*[len(o) - 1 for o in offs]):
        sl = tuple(slice(int(o[k]), int(o[k + 1])) for o, k in zip(offs, idx))
        r, g = ref[sl], got[sl]
        if r.size == 0:
            continue
        den = float(np.abs(r).max())
        if den == 0.0:
            den = gmax if gmax > 0.0 else 1.0
        worst = max(worst, float(np.abs(g - r).max()) / den)
    return worst


def site_parts(d, left, right):
    """Axis partition of a site tensor (d, m_left, m_right) for block_rel_err."""
    return [[1] * d, list(np.asarray(left["dim"] if isinstance(left, dict) else left.dim)),
            list(np.asarray(right["dim"] if isinstance(right, dict) else right.dim))]


def env_parts(w, bond):
    """Axis partition of an environment (w, m, m) for block_rel_err."""
    dims = list(np.asarray(bond["dim"] if isinstance(bond, dict) else bond.dim))
    return [[1] * w, dims, dims]


def site_to_dense(b, site):
    """Dense M[s, al, ar] of a device site tensor (via the library's block table)."""
    tab = site.blocks()
    flat = site.data.detach().cpu().numpy()
    blocks = b.unpack_blocks(tab, flat)
    spec = {"qp": site.qp.astype(np.int64), "left": _neutral(site.left),
            "right": _neutral(site.right), "blocks": blocks}
    return io.site_dense(spec)[0]


def env_to_dense(b, env):
    tab = env.blocks()
    blocks = b.unpack_blocks(tab, env.data.detach().cpu().numpy())
    spec = {"t": env.t.astype(np.int64), "bra": _neutral(env.bond), "ket": _neutral(env.bond),
            "blocks": blocks}
    return io.env_dense(spec)


def _neutral(bond):
    return {"q": bond.q.astype(np.int64), "dim": bond.dim.astype(np.int64)}


def fused_permutation(src, t, fused_q):
    """Dense positions (b * m + a, the oracle's fused order) listed in the fused-bond order.

    The fused bond has one sector per charge q + t[b] (ascending); inside a
    sector, channel b ascending, then the states of its source sector.
    """
    src_q, src_dim = src["q"], src["dim"]
    offs = np.concatenate([[0], np.cumsum(src_dim)])
    m = int(offs[-1])
    perm = []
    nsym = src_q.shape[1]
    for k in range(fused_q.shape[0]):
        for bch in range(t.shape[0]):
            if nsym == 0:
                j = 0
            else:
                hit = np.nonzero(np.all(src_q + t[bch][None, :] == fused_q[k][None, :], axis=1))[0]
                if len(hit) == 0:
                    continue
                j = int(hit[0])
            perm.extend(range(bch * m + offs[j], bch * m + offs[j] + src_dim[j]))
    return np.array(perm, dtype=np.int64)


# ---- problems ---------------------------------------------------------------------------

def problem(kind, seed, m_left=None, m_right=None, density=1.0):
    """Seeded local problem: bonds, envs (symmetric), W, a site tensor (neutral format)."""
    rng = si.rng_for(seed)
    if kind == "dense":
        ml, mr = m_left or 64, m_right or 64
        left, right = si.dense_bond(ml), si.dense_bond(mr)
        qp = np.zeros((2, 0), dtype=np.int64)
        t = np.zeros((5, 0), dtype=np.int64)
        idl, idr = (4,), (0,)
    elif kind == "u1":
        ml, mr = m_left or 150, m_right or 170
        left = si.gaussian_bond(ml, (1,), (3.0,), (2,), (5,))
        right = si.gaussian_bond(mr, (0,), (3.0,), (2,), (5,))
        qp, t = si.XXZ_QP, si.XXZ_T
        idl, idr = (4,), (0,)
    elif kind == "u1u1":
        ml, mr = m_left or 120, m_right or 130
        left = si.gaussian_bond(ml, (3, 1), (1.5, 1.5), (1, 2), (3, 3))
        right = si.gaussian_bond(mr, (4, 0), (1.5, 1.5), (1, 2), (3, 3))
        left = si._parity_filter(left, ml)
        right = si._parity_filter(right, mr)
        qp, t = si.HUB_QP, si.HUB_T
        idl, idr = (5,), (0,)
    elif kind in ("xxz_l100_m512_u1", "hubbard_l64_m1024_u1u1", "cylinder_4x16_m2048_u1"):
        left, right = si.central_bonds(kind, m=m_left)
        if kind.startswith("hubbard"):
            qp, t, idl, idr = si.HUB_QP, si.HUB_T, (5,), (0,)
        elif kind.startswith("cylinder"):
            qp = si.XXZ_QP
            t = np.array([[0]] + [[2], [-2], [0]] * 4 + [[0]], dtype=np.int64)
            idl, idr = (13,), (0,)
        else:
            qp, t, idl, idr = si.XXZ_QP, si.XXZ_T, (4,), (0,)
    else:
        raise KeyError(kind)
    Le = si.symmetric_env(rng, t, left, identity_channels=idl)
    Re = si.symmetric_env(rng, t, right, identity_channels=idr)
    W = si.random_mpo_site(rng, qp, t, t, density=density)
    A = si.random_site(rng, qp, left, right)
    return {"left": left, "right": right, "qp": qp, "t": t, "L": Le, "R": Re, "W": W, "A": A}
