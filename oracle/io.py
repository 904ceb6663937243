"""Conversion of the neutral block inputs into the oracle's dense arrays with labels.

Test infrastructure only (see the package docstring).  The neutral format is
described in ``seeded_inputs``: bonds are lists of charge sectors, tensors are
dictionaries of dense blocks.  The oracle embeds every block at its place in
a dense array (zeros elsewhere) and carries one charge label per index.
"""
import numpy as np


def bond_labels(bnd):
    q, dim = bnd["q"], bnd["dim"]
    return np.repeat(q, dim, axis=0).reshape(int(np.sum(dim)), q.shape[1])


def bond_offsets(bnd):
    return np.concatenate([[0], np.cumsum(bnd["dim"])]).astype(np.int64)


def site_dense(spec):
    """(M[s, al, ar], q_left, q_right) from a neutral site tensor."""
    ol, orr = bond_offsets(spec["left"]), bond_offsets(spec["right"])
    d = spec["qp"].shape[0]
    M = np.zeros((d, ol[-1], orr[-1]))
    for (s, i, j), blk in spec["blocks"].items():
        M[s, ol[i]:ol[i + 1], orr[j]:orr[j + 1]] = blk
    return M, bond_labels(spec["left"]), bond_labels(spec["right"])


def env_dense(spec):
    """E[b, a_bra, a_ket] from a neutral environment."""
    ob, ok = bond_offsets(spec["bra"]), bond_offsets(spec["ket"])
    w = spec["t"].shape[0]
    E = np.zeros((w, ob[-1], ok[-1]))
    for (b, ib, ik), blk in spec["blocks"].items():
        E[b, ob[ib]:ob[ib + 1], ok[ik]:ok[ik + 1]] = blk
    return E


def site_blocks(M, left, right, qp):
    """Cut a dense site tensor back into the neutral blocks of (left, right)."""
    ol, orr = bond_offsets(left), bond_offsets(right)
    out = {}
    for s in range(qp.shape[0]):
        for i in range(len(left["dim"])):
            for j in range(len(right["dim"])):
                if qp.shape[1] and not np.all(left["q"][i] + qp[s] == right["q"][j]):
                    continue
                out[(s, i, j)] = M[s, ol[i]:ol[i + 1], orr[j]:orr[j + 1]].copy()
    return out


def env_blocks(E, t, bra, ket):
    ob, ok = bond_offsets(bra), bond_offsets(ket)
    out = {}
    for b in range(t.shape[0]):
        for ib in range(len(bra["dim"])):
            for ik in range(len(ket["dim"])):
                if t.shape[1] and not np.all(ket["q"][ik] + t[b] == bra["q"][ib]):
                    continue
                out[(b, ib, ik)] = E[b, ob[ib]:ob[ib + 1], ok[ik]:ok[ik + 1]].copy()
    return out
