"""The contractions of the DMRG3S hot path, written as their definitions (oracle).

Test infrastructure only (see the package docstring).

Shapes: ``M[s, al, ar]`` (d, m_{i-1}, m_i); ``W[s_out, s_in, bl, br]``;
``L[b, a_bra, a_ket]``; ``R[b, a_bra, a_ket]``.  All arrays are float64.
"""
import numpy as np


def lw_a(L, W, M):
    """T2[br, s', al', ar] = sum_{bl, s, al} L[bl, al', al] W[s', s, bl, br] M[s, al, ar].

    The first two factors of the optimal ordering (((L M) W) R) of Sec. V:
    step 1 contracts L with M over the left MPS bond, step 2 multiplies in W
    over the physical index of M and the left MPO bond.
    """
    T1 = np.einsum("bXx,sxy->bsXy", L, M)          # step 1: L . M
    T2 = np.einsum("Ssbc,bsXy->cSXy", W, T1)       # step 2: . W
    return T2


def apply_heff(L, W, R, M):
    """HA[s', al', ar'] = sum L[bl, al', al] W[s', s, bl, br] M[s, al, ar] R[br, ar', ar].

    The left-hand side of the local eigenproblem L_{i-1} R_{i+1} W_i M_i = lambda M_i
    (Eq. es-iter, Sec. V), contracted in the order (((L M) W) R) (Sec. V);
    step 3 contracts R over the right MPO and MPS bonds.
    """
    T2 = lw_a(L, W, M)
    return np.einsum("cSXy,cYy->SXY", T2, R)       # step 3: . R


def apply_heff_literal(L, W, R, M):
    """The same contraction as one unordered sum (only for tiny shapes)."""
    return np.einsum("bXx,Ssbc,sxy,cYy->SXY", L, W, M, R, optimize=False)


def apply_heff_rows(L, W, R, M, rows):
    """HA[:, rows, :]: the definition of apply_heff for the listed left bra
    indices al' only (the same sum, restricted to those output rows), for
    sampled checks at sizes where the full product is too slow."""
    Lr = L[:, rows, :]                                   # (w_l, len(rows), m_l)
    T1 = np.einsum("bXx,sxy->bsXy", Lr, M)               # L . M
    T2 = np.einsum("Ssbc,bsXy->cSXy", W, T1)             # . W
    return np.einsum("cSXy,cYy->SXY", T2, R)             # . R


def expansion_term_lr(L, W, M, alpha):
    """P_i = alpha L_{i-1} M_i W_i in (d, m_{i-1}, w_i m_i)  (Eq. subexp-ourt, Sec. IV B).

    The fused right index is (br, ar) with br the slower index.
    """
    T2 = lw_a(L, W, M)                                 # (w_r, d, m_l, m_r)
    P = alpha * np.transpose(T2, (1, 2, 0, 3))          # (d, m_l, w_r, m_r)
    return P.reshape(P.shape[0], P.shape[1], -1)


def expansion_term_rl(R, W, M, alpha):
    """P_i = alpha R_{i+1} M_i W_i in (d, w_{i-1} m_{i-1}, m_i) for right-to-left sweeps (Sec. IV B).

    P[s', (bl, al), ar'] = alpha sum_{s, br, ar} W[s', s, bl, br] M[s, al, ar] R[br, ar', ar];
    the fused left index is (bl, al) with bl the slower index.
    """
    U1 = np.einsum("sxy,cYy->csxY", M, R)              # R . M over the right MPS bond
    U2 = np.einsum("Ssbc,csxY->SbxY", W, U1)           # . W over physical and right MPO bond
    P = alpha * U2
    return P.reshape(P.shape[0], -1, P.shape[3])


def left_env(Lprev, W, A):
    """L_i = L_{i-1} A_i^dagger W_i A_i  (Sec. II)."""
    T2 = lw_a(Lprev, W, A)                             # [c, s', X, y]
    return np.einsum("SXY,cSXy->cYy", A.conj(), T2)


def right_env(Rnext, W, B):
    """R_i = R_{i+1} B_i^dagger W_i B_i  (Sec. II), contracted as the mirror of left_env."""
    U1 = np.einsum("sxy,cYy->csxY", B, Rnext)          # B . R over the right MPS bond
    U2 = np.einsum("Ssbc,csxY->SbxY", W, U1)           # . W
    return np.einsum("SXY,SbxY->bXx", B.conj(), U2)    # . B^dagger


def expectation(L, W, R, M):
    """<Psi|H|Psi> = L_{i-1} M_i^dagger W_i M_i R_{i+1}  (Sec. II)."""
    return float(np.vdot(M, apply_heff(L, W, R, M)))


def rayleigh(L, W, R, M):
    """Energy of the (not necessarily normalised) centre tensor M."""
    return expectation(L, W, R, M) / float(np.vdot(M, M))


def mpo_gradient(L, R, M):
    """G[s', s, bl, br] = sum L[bl, al', al] M*[s', al', ar'] M[s, al, ar] R[br, ar', ar].

    d<Psi|H|Psi>/dW_i[s', s, bl, br] at fixed MPS: the network of Sec. II with
    W_i taken out.  Divided by <Psi|Psi> it gives the Hellmann-Feynman
    derivative of the energy with respect to the entries of W_i.
    """
    # the same sum, associated pairwise (a single four-operand einsum falls back
    # to the naive loop over all eight indices at large m)
    T1 = np.einsum("bXx,sxy->bsXy", L, M)              # ket copy of M through L
    Y = np.einsum("SXY,cYy->ScXy", M.conj(), R)        # bra copy of M through R
    return np.einsum("bsXy,ScXy->Ssbc", T1, Y)
