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
