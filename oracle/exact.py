"""Exact ground-state energies used to pin the oracle, oracle side.

Test infrastructure only (see the package docstring).

* ``ed_ground_energy``: dense diagonalisation of a Hamiltonian restricted to a
  charge sector (numpy ``eigvalsh``);
* ``ed_sparse_spin``: Lanczos-free sparse diagonalisation (scipy ``eigsh``) of
  a spin-1/2 bond Hamiltonian in a fixed-S^z sector, built from bit
  operations without any MPO;
* ``xx_chain_energy`` / ``free_fermion_energy``: Jordan-Wigner closed forms of
  the open XX chain and the U=0 Hubbard chain.  Single-particle energies of an
  open chain with hopping amplitude h are 2h cos(pi k/(l+1)), k = 1..l.
"""
import numpy as np


def ed_ground_energy(H, charges=None, target=None):
    """Smallest eigenvalue of H, optionally inside the sector ``charges == target``."""
    if charges is not None:
        sel = np.all(charges == np.asarray(target)[None, :], axis=1)
        H = H[np.ix_(sel, sel)]
    return float(np.linalg.eigvalsh(H)[0])


def xx_chain_energy(L, J=1.0):
    """Open XX chain J sum (SxSx + SySy): free fermions with hopping J/2."""
    k = np.arange(1, L + 1)
    eps = J * np.cos(np.pi * k / (L + 1))
    return float(np.sum(eps[eps < 0]))


def free_fermion_energy(L, n_up, n_dn, t_hop=1.0):
    """Open U=0 Hubbard chain: fill the lowest single-particle levels per spin."""
    k = np.arange(1, L + 1)
    eps = np.sort(-2.0 * t_hop * np.cos(np.pi * k / (L + 1)))
    return float(np.sum(eps[:n_up]) + np.sum(eps[:n_dn]))


def ed_sparse_spin(L, bonds, two_sz=0):
    """Ground energy of a spin-1/2 bond Hamiltonian in the 2*S^z = two_sz sector."""
    import itertools
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n_up = (L + two_sz) // 2
    states = []
    for ups in itertools.combinations(range(L), n_up):
        s = 0
        for u in ups:
            s |= 1 << u
        states.append(s)
    states = np.array(sorted(states), dtype=np.int64)
    index = {int(s): n for n, s in enumerate(states)}
    rows, cols, vals = [], [], []
    diag = np.zeros(len(states))
    for (i, j, jxy, jz) in bonds:
        bi = (states >> i) & 1
        bj = (states >> j) & 1
        diag += jz * np.where(bi == bj, 0.25, -0.25)
        flip = np.nonzero(bi != bj)[0]
        for n in flip:
            s2 = int(states[n]) ^ ((1 << i) | (1 << j))
            rows.append(index[s2])
            cols.append(n)
            vals.append(0.5 * jxy)
    n = len(states)
    H = sp.csr_matrix((vals, (rows, cols)), shape=(n, n)) + sp.diags(diag)
    w = sla.eigsh(H, k=1, which="SA", tol=1e-13, maxiter=100000)[0]
    return float(w[0])


def ed_sparse_spin_s(L, bonds, two_s, two_sz=0):
    """Ground energy of a spin-S bond Hamiltonian (S = two_s / 2) in the
    2 S^z_total = two_sz sector: sum over bonds (i, j, Jxy, Jz) of
    Jxy/2 (S+_i S-_j + S-_i S+_j) + Jz Sz_i Sz_j.  Basis states are integers in
    base d = two_s + 1 (site 0 the most significant digit, digit k meaning
    m = S - k), the order of the Kronecker-product Hamiltonians."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    d = two_s + 1
    S = two_s / 2.0
    allidx = np.arange(d ** L, dtype=np.int64)
    digits = np.stack([(allidx // d ** (L - 1 - i)) % d for i in range(L)])   # (L, d^L)
    keep = digits.sum(0) * 2 == L * two_s - two_sz
    states, dig = allidx[keep], digits[:, keep]
    m = S - dig                                                             # (L, n)
    n = len(states)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for (i, j, jxy, jz) in bonds:
        diag += jz * m[i] * m[j]
        # S+_i S-_j: m_i -> m_i + 1 (digit k_i - 1), m_j -> m_j - 1 (digit k_j + 1)
        ok = (dig[i] >= 1) & (dig[j] <= two_s - 1)
        src = np.nonzero(ok)[0]
        amp = np.sqrt(S * (S + 1) - m[i, src] * (m[i, src] + 1)) * \
            np.sqrt(S * (S + 1) - m[j, src] * (m[j, src] - 1))
        dst_state = states[src] - d ** (L - 1 - i) + d ** (L - 1 - j)
        dst = np.searchsorted(states, dst_state)
        rows += [dst, src]
        cols += [src, dst]
        vals += [0.5 * jxy * amp, 0.5 * jxy * amp]
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)) + sp.diags(diag)
    if n <= 64:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    w = sla.eigsh(H, k=1, which="SA", tol=1e-13, maxiter=100000)[0]
    return float(w[0])
