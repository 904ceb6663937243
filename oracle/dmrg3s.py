"""DMRG3S (strictly single-site DMRG with subspace expansion), oracle side.

Test infrastructure only (see the package docstring).

The local update follows the eight steps listed in Sec. V in their order:
(1) eigensolver for the smallest eigenpair of Eq. es-iter, (2) expansion term
alpha P_i of Eq. subexp-ourt, (3) subspace expansion of M_i and zero padding of
the neighbour (Sec. IV A), (4) SVD and truncation, (5) S V^dagger multiplied
into the neighbour, (6) new environment, (7) energy after truncation and the
adaptive mixing factor (Sec. VI), (8) move on.

Readings of points the paper leaves open (each is a documented choice):

* eigensolver: Lanczos with full classical Gram-Schmidt reorthogonalisation
  applied twice (CGS2), started from the current site tensor;
* truncation keeps ``min(m_max, #{s > 1e-12 s_max})`` singular values, ordered
  by (-s, charge sector, index inside the sector); 1e-12 s_max is the
  numerical zero of an FP64 SVD (rounding noise of the factorisation sits
  near 1e-14 s_max and must not be kept as states);
* the energy after truncation is the Rayleigh quotient of the neighbour
  tensor (it is not normalised after step 5) with the environments of the
  neighbour site;
* alpha rule: with dE_O = lambda* - E_in (<= 0) and dE_T = E_f - lambda*, and
  r = dE_T / |dE_O|: if |dE_O| < 1e-13 |E| shrink; elif dE_T < 0 or r < 0.3
  grow; elif r > 1 shrink twice; else shrink (grow = x1.25, shrink = x0.8),
  clamped to [alpha_min, alpha_max];
* a sweep is one right-to-left pass (sites l..2) followed by one
  left-to-right pass (sites 1..l-1); a run stops when the relative energy
  change between two sweeps drops below ``conv_tol``.
"""
from dataclasses import dataclass, field

import numpy as np

from . import contract
from .labels import combine, sectors


# ---- eigensolver ------------------------------------------------------------

def lanczos_ground(matvec, x0, kmax=40, tol=1e-10, beta_tol=1e-14):
    """Smallest eigenpair of a symmetric operator by Lanczos with CGS2.

    Returns (theta, x, iterations).  Stops when the Ritz residual
    |beta_k y_k| <= tol * max(1, |theta|), when beta_k < beta_tol (invariant
    subspace) or after kmax matrix-vector products.
    """
    shape = x0.shape
    v = x0.reshape(-1).astype(np.float64)
    nrm = np.linalg.norm(v)
    if nrm == 0.0:
        raise ValueError("zero start vector")
    V = [v / nrm]
    alphas, betas = [], []
    theta, y = None, None
    for k in range(kmax):
        w = matvec(V[k].reshape(shape)).reshape(-1)
        a = float(np.dot(V[k], w))
        alphas.append(a)
        Vm = np.array(V)
        for _ in range(2):                        # CGS2 against all previous vectors
            w = w - Vm.T @ (Vm @ w)
        b = float(np.linalg.norm(w))
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        evals, evecs = np.linalg.eigh(T)
        theta, y = float(evals[0]), evecs[:, 0]
        resid = abs(b * y[-1])
        if resid <= tol * max(1.0, abs(theta)) or b < beta_tol or k + 1 == kmax:
            break
        betas.append(b)
        V.append(w / b)
    x = np.array(V[: len(y)]).T @ y
    x /= np.linalg.norm(x)
    return theta, x.reshape(shape), len(alphas)


# ---- SVD truncation (Sec. IV A, steps 4 and 5 of Sec. V) ----------------------

def _ordered_keep(svals, m_max, eps):
    """(sector, index) pairs kept, ordered by (-s, sector, index)."""
    cand = []
    for sec, s in enumerate(svals):
        for j, v in enumerate(s):
            cand.append((-float(v), sec, j))
    if not cand:
        return []
    smax = -min(c[0] for c in cand)
    cand.sort()
    keep = [(sec, j) for (negs, sec, j) in cand if -negs > eps * smax]
    return keep[:m_max]


def truncate_lr(Mt, qphys, ql, qr, m_max, eps=1e-12):
    """SVD of Mt reshaped to ((s, al), ar) per charge sector; keep m_max states.

    Returns (A, SV, q_new): A (d, m_l, k) left-normalised, SV (k, m_r) = S V^dagger.
    """
    d, ml, mr = Mt.shape
    X = Mt.reshape(d * ml, mr)
    rowq = combine(qphys, ql)
    secs, svals, facs = [], [], []
    for key, cols in sectors(qr):
        if qr.shape[1] == 0:
            rows = np.arange(d * ml)
        else:
            rows = np.nonzero(np.all(rowq == np.array(key)[None, :], axis=1))[0]
        if len(rows) == 0:
            continue
        U, S, Vt = np.linalg.svd(X[np.ix_(rows, cols)], full_matrices=False)
        secs.append((key, rows, cols))
        svals.append(S)
        facs.append((U, S, Vt))
    keep = _ordered_keep(svals, m_max, eps)
    k = len(keep)
    A = np.zeros((d * ml, k))
    SV = np.zeros((k, mr))
    qn = np.zeros((k, qr.shape[1]), dtype=np.int64)
    for n, (sec, j) in enumerate(keep):
        key, rows, cols = secs[sec]
        U, S, Vt = facs[sec]
        A[rows, n] = U[:, j]
        SV[n, cols] = S[j] * Vt[j, :]
        qn[n, :] = key
    return A.reshape(d, ml, k), SV, qn


def truncate_rl(Mt, qphys, ql, qr, m_max, eps=1e-12):
    """SVD of Mt reshaped to (al, (s, ar)) per charge sector; keep m_max states.

    Returns (B, US, q_new): B (d, k, m_r) right-normalised, US (m_l, k) = U S.
    """
    d, ml, mr = Mt.shape
    X = np.transpose(Mt, (1, 0, 2)).reshape(ml, d * mr)
    colq = combine(-qphys, qr)
    secs, svals, facs = [], [], []
    for key, rows in sectors(ql):
        if ql.shape[1] == 0:
            cols = np.arange(d * mr)
        else:
            cols = np.nonzero(np.all(colq == np.array(key)[None, :], axis=1))[0]
        if len(cols) == 0:
            continue
        U, S, Vt = np.linalg.svd(X[np.ix_(rows, cols)], full_matrices=False)
        secs.append((key, rows, cols))
        svals.append(S)
        facs.append((U, S, Vt))
    keep = _ordered_keep(svals, m_max, eps)
    k = len(keep)
    Bm = np.zeros((k, d * mr))
    US = np.zeros((ml, k))
    qn = np.zeros((k, ql.shape[1]), dtype=np.int64)
    for n, (sec, j) in enumerate(keep):
        key, rows, cols = secs[sec]
        U, S, Vt = facs[sec]
        Bm[n, cols] = Vt[j, :]
        US[rows, n] = U[:, j] * S[j]
        qn[n, :] = key
    B = np.transpose(Bm.reshape(k, d, mr), (1, 0, 2))
    return B, US, qn


# ---- mixing factor (Sec. VI) ------------------------------------------------

@dataclass
class AlphaRule:
    alpha0: float = 1e-2
    target: float = 0.3
    up: float = 1.25
    down: float = 0.8
    alpha_min: float = 1e-14
    alpha_max: float = 1.0
    fixed: bool = False

    def update(self, alpha, e_in, lam, e_f):
        if self.fixed:
            return alpha
        d_o = lam - e_in
        d_t = e_f - lam
        if abs(d_o) < 1e-13 * max(abs(lam), 1e-300):
            alpha *= self.down
        elif d_t < 0.0 or d_t / abs(d_o) < self.target:
            alpha *= self.up
        elif d_t / abs(d_o) > 1.0:
            alpha *= self.down * self.down
        else:
            alpha *= self.down
        return min(max(alpha, self.alpha_min), self.alpha_max)


# ---- MPS state ----------------------------------------------------------------

@dataclass
class MPS:
    M: list                 # site tensors (d, m_{i-1}, m_i)
    q: list                 # bond labels q[0..l], each (m_i, nsym)
    qphys: np.ndarray       # (d, nsym)

    @property
    def L(self):
        return len(self.M)


def left_normalise(tensors):
    """QR sweep from the left; the norm ends up in the last tensor, then divided out."""
    out = []
    carry = np.ones((1, 1))
    for n, M in enumerate(tensors):
        M = np.einsum("xy,syz->sxz", carry, M)
        d, ml, mr = M.shape
        if n == len(tensors) - 1:
            out.append(M / np.linalg.norm(M))
            break
        X = M.reshape(d * ml, mr)
        Q, Rm = np.linalg.qr(X)
        k = Q.shape[1]
        out.append(Q.reshape(d, ml, k))
        carry = Rm
    return out


def right_normalise(tensors):
    """QR sweep from the right (LQ of each site); the norm ends up in the first tensor."""
    out = [None] * len(tensors)
    carry = np.ones((1, 1))
    for n in range(len(tensors) - 1, -1, -1):
        M = np.einsum("sxy,yz->sxz", tensors[n], carry)
        d, ml, mr = M.shape
        if n == 0:
            out[0] = M / np.linalg.norm(M)
            break
        X = np.transpose(M, (1, 0, 2)).reshape(ml, d * mr)
        Q, Rm = np.linalg.qr(X.T)               # X = Rm^T Q^T
        k = Q.shape[1]
        out[n] = np.transpose(Q.T.reshape(k, d, mr), (1, 0, 2))
        carry = Rm.T
    return out


def product_state(qphys, local_states):
    """m = 1 product state; bond labels accumulate the local charges from the left."""
    d, nsym = qphys.shape
    M, q = [], [np.zeros((1, nsym), dtype=np.int64)]
    for s in local_states:
        T = np.zeros((d, 1, 1))
        T[s, 0, 0] = 1.0
        M.append(T)
        q.append(q[-1] + qphys[s][None, :])
    return MPS(M, q, qphys.copy())


def mps_to_dense(mps):
    psi = mps.M[0][:, 0, :]
    for T in mps.M[1:]:
        psi = np.einsum("Pa,sab->Psb", psi, T).reshape(-1, T.shape[2])
    return psi[:, 0]


# ---- environments -----------------------------------------------------------------

def build_left_envs(mpo, mps, upto):
    Ls = [np.ones((1, 1, 1))]
    for i in range(upto):
        Ls.append(contract.left_env(Ls[-1], mpo.W[i], mps.M[i]))
    return Ls


def build_right_envs(mpo, mps, downto):
    """Right environments R[i] of everything right of site i, for i >= downto."""
    L = mps.L
    Rs = {L - 1: np.ones((1, 1, 1))}
    for i in range(L - 1, downto, -1):
        Rs[i - 1] = contract.right_env(Rs[i], mpo.W[i], mps.M[i])
    return Rs


# ---- sweeps -----------------------------------------------------------------------

@dataclass
class SweepOptions:
    m_max: int = 64
    max_sweeps: int = 6
    conv_tol: float = 1e-9
    lanczos_kmax: int = 40
    lanczos_tol: float = 1e-10
    trunc_eps: float = 1e-12
    alpha: AlphaRule = field(default_factory=AlphaRule)


@dataclass
class SweepLog:
    energies: list = field(default_factory=list)      # energy after every sweep
    alphas: list = field(default_factory=list)        # alpha after every local update
    lambdas: list = field(default_factory=list)       # eigensolver values, in order
    bond_dims: list = field(default_factory=list)
    converged: bool = False


class DMRG3S:
    """Driver holding the MPS and the environments of a mixed-canonical state."""

    def __init__(self, mpo, mps, opts, left_env=None, right_env=None, centre=None):
        """``left_env`` / ``right_env`` replace the trivial boundaries L_0 = R_{l+1} = 1
        (a window of a longer chain); ``centre`` is the orthogonality centre (default l)."""
        self.mpo, self.mps, self.opts = mpo, mps, opts
        self.alpha = opts.alpha.alpha0
        L = mps.L
        centre = L - 1 if centre is None else centre
        self.Lenv = {0: np.ones((1, 1, 1)) if left_env is None else left_env}
        for i in range(centre):
            self.Lenv[i + 1] = contract.left_env(self.Lenv[i], mpo.W[i], mps.M[i])
        self.Renv = {L - 1: np.ones((1, 1, 1)) if right_env is None else right_env}
        for i in range(L - 1, centre, -1):
            self.Renv[i - 1] = contract.right_env(self.Renv[i], mpo.W[i], mps.M[i])
        self.e_in = contract.rayleigh(self.Lenv[centre], mpo.W[centre], self.Renv[centre],
                                      mps.M[centre])

    def _eig(self, i):
        Le, Re, W = self.Lenv[i], self.Renv[i], self.mpo.W[i]
        lam, x, _ = lanczos_ground(lambda v: contract.apply_heff(Le, W, Re, v), self.mps.M[i],
                                   kmax=self.opts.lanczos_kmax, tol=self.opts.lanczos_tol)
        return lam, x

    def update_lr(self, i):
        """Local update of site i during a left-to-right sweep (steps 1-8, Sec. V)."""
        mps, mpo, o = self.mps, self.mpo, self.opts
        lam, Mstar = self._eig(i)                                           # 1
        P = contract.expansion_term_lr(self.Lenv[i], mpo.W[i], Mstar, self.alpha)   # 2
        Mt = np.concatenate([Mstar, P], axis=2)                             # 3
        qr_t = np.concatenate([mps.q[i + 1], combine(mpo.t[i + 1], mps.q[i + 1])], axis=0)
        A, SV, qn = truncate_lr(Mt, mps.qphys, mps.q[i], qr_t, o.m_max, o.trunc_eps)   # 4
        mr = mps.M[i].shape[2]
        Bn = np.einsum("kx,sxy->sky", SV[:, :mr], mps.M[i + 1])              # 5
        mps.M[i], mps.M[i + 1], mps.q[i + 1] = A, Bn, qn
        self.Lenv[i + 1] = contract.left_env(self.Lenv[i], mpo.W[i], A)     # 6
        e_f = contract.rayleigh(self.Lenv[i + 1], mpo.W[i + 1], self.Renv[i + 1], Bn)  # 7
        self.alpha = o.alpha.update(self.alpha, self.e_in, lam, e_f)
        self.e_in = e_f
        return lam, e_f

    def update_rl(self, i):
        """Local update of site i during a right-to-left sweep (mirror of update_lr)."""
        mps, mpo, o = self.mps, self.mpo, self.opts
        lam, Mstar = self._eig(i)
        P = contract.expansion_term_rl(self.Renv[i], mpo.W[i], Mstar, self.alpha)
        Mt = np.concatenate([Mstar, P], axis=1)
        ql_t = np.concatenate([mps.q[i], combine(mpo.t[i], mps.q[i])], axis=0)
        B, US, qn = truncate_rl(Mt, mps.qphys, ql_t, mps.q[i + 1], o.m_max, o.trunc_eps)
        ml = mps.M[i].shape[1]
        An = np.einsum("sxy,yk->sxk", mps.M[i - 1], US[:ml, :])
        mps.M[i], mps.M[i - 1], mps.q[i] = B, An, qn
        self.Renv[i - 1] = contract.right_env(self.Renv[i], mpo.W[i], B)
        e_f = contract.rayleigh(self.Lenv[i - 1], mpo.W[i - 1], self.Renv[i - 1], An)
        self.alpha = o.alpha.update(self.alpha, self.e_in, lam, e_f)
        self.e_in = e_f
        return lam, e_f

    def sweep(self, log):
        L = self.mps.L
        e = None
        for i in range(L - 1, 0, -1):
            lam, e = self.update_rl(i)
            log.lambdas.append(lam)
            log.alphas.append(self.alpha)
        for i in range(0, L - 1):
            lam, e = self.update_lr(i)
            log.lambdas.append(lam)
            log.alphas.append(self.alpha)
        log.bond_dims.append([T.shape[2] for T in self.mps.M[:-1]])
        return e

    def run(self):
        log = SweepLog()
        for _ in range(self.opts.max_sweeps):
            e = self.sweep(log)
            log.energies.append(e)
            if len(log.energies) >= 2:
                prev = log.energies[-2]
                if abs(e - prev) / abs(e) < self.opts.conv_tol:
                    log.converged = True
                    break
        return log
