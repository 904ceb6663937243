"""Charge labels for abelian (U(1) or U(1)xU(1)) symmetries, oracle side.

Test infrastructure only (see the package docstring).

A basis of dimension ``n`` carries an integer array ``q`` of shape ``(n, nsym)``
with one charge vector per basis state; ``nsym == 0`` means no symmetry.  The
selection rules follow from charge conservation (Sec. II and Sec. III A of the
paper, where a state "transforms as" a quantum number):

* MPS tensor ``M[s, al, ar]`` may be non-zero only if
  ``q_r[ar] == q_l[al] + q_phys[s]`` (the right basis counts the charge of all
  sites up to and including site i);
* MPO tensor ``W[s_out, s_in, bl, br]`` only if
  ``q_phys[s_out] - q_phys[s_in] + t_l[bl] == t_r[br]`` (an MPO channel carries
  the charge the operators placed to its left have added);
* environments ``L[b, a_bra, a_ket]`` and ``R[b, a_bra, a_ket]`` only if
  ``q[a_bra] == q[a_ket] + t[b]``.
"""
import numpy as np


def as_labels(q, n=None, nsym=None):
    q = np.asarray(q, dtype=np.int64)
    if q.ndim == 1:
        q = q.reshape(-1, 1) if (nsym is None or nsym == 1) else q.reshape(n, nsym)
    if n is not None:
        assert q.shape[0] == n
    return q


def site_mask(qp, ql, qr):
    """Boolean mask of the entries of M[s, al, ar] allowed by charge conservation."""
    if qp.shape[1] == 0:
        return np.ones((qp.shape[0], ql.shape[0], qr.shape[0]), dtype=bool)
    tot = qp[:, None, None, :] + ql[None, :, None, :]
    return np.all(tot == qr[None, None, :, :], axis=-1)


def env_mask(t, qbra, qket):
    """Mask of L[b, a_bra, a_ket] (or R) allowed by charge conservation."""
    if t.shape[1] == 0:
        return np.ones((t.shape[0], qbra.shape[0], qket.shape[0]), dtype=bool)
    tot = qket[None, None, :, :] + t[:, None, None, :]
    return np.all(tot == qbra[None, :, None, :], axis=-1)


def mpo_mask(qp, tl, tr):
    """Mask of W[s_out, s_in, bl, br] allowed by charge conservation."""
    if qp.shape[1] == 0:
        return np.ones((qp.shape[0], qp.shape[0], tl.shape[0], tr.shape[0]), dtype=bool)
    lhs = (qp[:, None, None, None, :] - qp[None, :, None, None, :]
           + tl[None, None, :, None, :])
    return np.all(lhs == tr[None, None, None, :, :], axis=-1)


def combine(q_outer, q_inner):
    """Labels of a fused index (outer-major) whose charge is the sum of both parts."""
    out = q_outer[:, None, :] + q_inner[None, :, :]
    return out.reshape(q_outer.shape[0] * q_inner.shape[0], q_outer.shape[1])


def sectors(q):
    """Distinct charge vectors of a basis, in lexicographic order, with the member indices."""
    if q.shape[1] == 0:
        return [((), np.arange(q.shape[0]))]
    keys = sorted({tuple(int(v) for v in row) for row in q})
    out = []
    for k in keys:
        idx = np.nonzero(np.all(q == np.array(k)[None, :], axis=1))[0]
        out.append((k, idx))
    return out
