"""Hamiltonians as MPOs and as dense matrices, oracle side.

Test infrastructure only (see the package docstring).

Two independent routes are kept on purpose:

* ``mpo_*`` builds the site tensors ``W_i[s_out, s_in, bl, br]`` of Sec. II (a
  rank-4 tensor per site, ``H = W_1 ... W_l``) with a lower-triangular
  finite-state layout: channel 0 means "all terms finished", the last channel
  means "nothing placed yet"; the left boundary row is the last channel and
  the right boundary column is channel 0;
* ``dense_*`` builds the same Hamiltonian directly from Kronecker products
  (and, for fermions, a Jordan-Wigner string over 2l modes), never touching
  the MPO code.  ``mpo_to_dense`` contracts an MPO into a matrix so the two
  routes can be compared entry by entry.

Spin-1/2 local basis: index 0 = up, 1 = down, charge 2*S^z in {+1, -1}.
Spin-S local basis (``two_s`` = 2S): index k holds m = S - k, charge 2m.
Fermion (Hubbard) local basis: index 2*n_up + n_dn, i.e. 0=|0>, 1=|dn>,
2=|up>, 3=|up dn>; charges (N, 2*S^z).  Mode order for the Jordan-Wigner
string: site-major, spin-up before spin-down.
"""
import numpy as np

# ---- local operators ------------------------------------------------------

SZ = np.diag([0.5, -0.5])
SP = np.array([[0.0, 1.0], [0.0, 0.0]])   # <up|S+|dn> = 1
SM = SP.T.copy()
I2 = np.eye(2)
SPIN_HALF_Q = np.array([[1], [-1]])       # 2*S^z of (up, dn)

_ANN = np.array([[0.0, 1.0], [0.0, 0.0]])  # a|1> = |0> in the (|0>,|1>) basis
_PAR = np.diag([1.0, -1.0])               # (-1)^n
A_UP = np.kron(_ANN, I2)
A_DN = np.kron(_PAR, _ANN)
F_PAR = np.kron(_PAR, _PAR)
N_UP = A_UP.T @ A_UP
N_DN = A_DN.T @ A_DN
I4 = np.eye(4)
HUB_Q = np.array([[0, 0], [1, -1], [1, 1], [2, 0]])   # (N, 2Sz) of 0,dn,up,updn


def spin_ops(two_s):
    """(S+, S-, Sz, identity, charges) of spin S = two_s / 2 in the basis
    m = S, S-1, ..., -S: <m+1|S+|m> = sqrt(S(S+1) - m(m+1)), charge 2m."""
    d = two_s + 1
    S = two_s / 2.0
    m = S - np.arange(d)
    sp = np.zeros((d, d))
    for k in range(1, d):          # |m = S - k> -> |m + 1> (index k - 1)
        sp[k - 1, k] = np.sqrt(S * (S + 1) - m[k] * (m[k] + 1))
    q = (two_s - 2 * np.arange(d)).reshape(d, 1)
    return sp, sp.T.copy(), np.diag(m), np.eye(d), q


class MPO:
    """List of W tensors plus the charge labels of every MPO bond."""

    def __init__(self, W, qphys, t):
        self.W = W            # list of (d, d, w_{i-1}, w_i)
        self.qphys = qphys    # (d, nsym)
        self.t = t            # list of l+1 arrays (w_i, nsym); t[0], t[l] are the boundaries

    @property
    def L(self):
        return len(self.W)


def _lower_triangular_chain(L, bulk, t):
    """Slice a bulk W (d, d, w, w) into first row / last column for an open chain."""
    w = bulk.shape[2]
    Ws = []
    for i in range(L):
        Wi = bulk.copy()
        tl, tr = t, t
        if i == 0:
            Wi = Wi[:, :, w - 1:w, :]
            tl = t[w - 1:w]
        if i == L - 1:
            Wi = Wi[:, :, :, 0:1]
            tr = t[0:1]
        Ws.append(Wi)
    ts = [t[w - 1:w]] + [t] * (L - 1) + [t[0:1]]
    return Ws, ts


def mpo_xxz(L, J=1.0, Delta=1.0):
    """S=1/2 XXZ chain, open BC: H = J sum_i [ (S+S- + S-S+)/2 + Delta Sz Sz ]  (w = 5).

    Channels: 0 done, 1 holds S- (closes with S+), 2 holds S+ (closes with S-),
    3 holds Sz, 4 nothing placed yet.  Charges t in units of 2*S^z.
    """
    d, w = 2, 5
    Wb = np.zeros((d, d, w, w))
    Wb[:, :, 0, 0] = I2
    Wb[:, :, 1, 0] = SP
    Wb[:, :, 2, 0] = SM
    Wb[:, :, 3, 0] = SZ
    Wb[:, :, 4, 1] = 0.5 * J * SM
    Wb[:, :, 4, 2] = 0.5 * J * SP
    Wb[:, :, 4, 3] = J * Delta * SZ
    Wb[:, :, 4, 4] = I2
    t = np.array([[0], [-2], [2], [0], [0]])
    Ws, ts = _lower_triangular_chain(L, Wb, t)
    return MPO(Ws, SPIN_HALF_Q.copy(), ts)


def mpo_hubbard(L, t_hop=1.0, U=0.0):
    """1-D Fermi-Hubbard chain, open BC (w = 6):
    H = -t sum_{i,s} (c+_{i s} c_{i+1 s} + h.c.) + U sum_i n_{i up} n_{i dn}.

    With the Jordan-Wigner string, c+_i c_{i+1} = (a+ F)_i (a)_{i+1} and
    c+_{i+1} c_i = (F a)_i (a+)_{i+1}.  Channels: 0 done, 1 holds a+_up F,
    2 holds F a_up, 3 holds a+_dn F, 4 holds F a_dn, 5 nothing placed yet.
    """
    d, w = 4, 6
    Wb = np.zeros((d, d, w, w))
    Wb[:, :, 0, 0] = I4
    Wb[:, :, 1, 0] = A_UP
    Wb[:, :, 2, 0] = A_UP.T
    Wb[:, :, 3, 0] = A_DN
    Wb[:, :, 4, 0] = A_DN.T
    Wb[:, :, 5, 0] = U * (N_UP @ N_DN)
    Wb[:, :, 5, 1] = -t_hop * (A_UP.T @ F_PAR)
    Wb[:, :, 5, 2] = -t_hop * (F_PAR @ A_UP)
    Wb[:, :, 5, 3] = -t_hop * (A_DN.T @ F_PAR)
    Wb[:, :, 5, 4] = -t_hop * (F_PAR @ A_DN)
    Wb[:, :, 5, 5] = I4
    t = np.array([[0, 0], [1, 1], [-1, -1], [1, -1], [-1, 1], [0, 0]])
    Ws, ts = _lower_triangular_chain(L, Wb, t)
    return MPO(Ws, HUB_Q.copy(), ts)


def mpo_spin_bonds(L, bonds, two_s=1):
    """Spin-S Heisenberg-type MPO (S = two_s / 2) for arbitrary two-site couplings.

    ``bonds`` is a list of ``(i, j, Jxy, Jz)`` with 0 <= i < j < L meaning
    ``Jxy/2 (S+_i S-_j + S-_i S+_j) + Jz Sz_i Sz_j``.  Finite-state layout: at
    each MPO bond, channel 0 = done, last = nothing placed, and three channels
    (S+, S-, Sz placed) for every site left of the bond with a partner right of
    it.  This is the construction used for the cylinder of the benchmark
    suite; for nearest-neighbour bonds it reproduces ``mpo_xxz``'s w = 5.
    """
    partners = {}
    sp, sm, sz, eye, qphys = spin_ops(two_s)
    d = two_s + 1
    for (i, j, jxy, jz) in bonds:
        assert 0 <= i < j < L
        partners.setdefault(i, []).append((j, jxy, jz))
    # channel lists per MPO bond index k = 0..L (bond k sits left of site k)
    chans = []
    for k in range(L + 1):
        sites = sorted({i for (i, j, _, _) in bonds if i < k <= j})
        ch = [("done",)]
        for s in sites:
            ch += [(s, "S+"), (s, "S-"), (s, "Sz")]
        ch.append(("start",))
        chans.append(ch)
    chans[0] = [("start",)]
    chans[L] = [("done",)]
    qmap = {"S+": 2, "S-": -2, "Sz": 0}
    opmap = {"S+": sp, "S-": sm, "Sz": sz}
    close = {"S+": ("S-", 0.5), "S-": ("S+", 0.5), "Sz": ("Sz", None)}
    Ws, ts = [], []
    for k in range(L + 1):
        ts.append(np.array([[0] if c[0] in ("done", "start") else [qmap[c[1]]] for c in chans[k]]))
    for site in range(L):
        cl, cr = chans[site], chans[site + 1]
        ixl = {c: n for n, c in enumerate(cl)}
        ixr = {c: n for n, c in enumerate(cr)}
        Wi = np.zeros((d, d, len(cl), len(cr)))
        if ("done",) in ixl and ("done",) in ixr:
            Wi[:, :, ixl[("done",)], ixr[("done",)]] += eye
        if ("start",) in ixl and ("start",) in ixr:
            Wi[:, :, ixl[("start",)], ixr[("start",)]] += eye
        # open new channels at this site
        if ("start",) in ixl:
            for op in ("S+", "S-", "Sz"):
                if (site, op) in ixr:
                    Wi[:, :, ixl[("start",)], ixr[(site, op)]] += opmap[op]
        # carry or close open channels
        for c in cl:
            if c[0] in ("done", "start"):
                continue
            src, op = c
            if c in ixr:
                Wi[:, :, ixl[c], ixr[c]] += eye
            for (j, jxy, jz) in partners.get(src, []):
                if j == site:
                    cop, half = close[op]
                    coef = jxy * half if half is not None else jz
                    Wi[:, :, ixl[c], ixr[("done",)]] += coef * opmap[cop]
        Ws.append(Wi)
    return MPO(Ws, qphys, ts)


def cylinder_bonds(Lx, Ly, J=1.0):
    """Nearest-neighbour bonds of an Lx x Ly cylinder (periodic in y), snake order.

    Site (x, y) sits at chain index x*Ly + (y if x even else Ly-1-y).
    """
    def idx(x, y):
        return x * Ly + (y if x % 2 == 0 else Ly - 1 - y)
    bonds = set()
    for x in range(Lx):
        for y in range(Ly):
            nbrs = [(x, (y + 1) % Ly)]
            if x + 1 < Lx:
                nbrs.append((x + 1, y))
            for (x2, y2) in nbrs:
                a, b = idx(x, y), idx(x2, y2)
                if a != b:
                    bonds.add((min(a, b), max(a, b)))
    return [(i, j, J, J) for (i, j) in sorted(bonds)]


def mpo_two_spin_example():
    """The two-site MPO printed in the subspace-expansion example (Sec. IV C).

    Taken exactly as printed: W_1 = [S+/sqrt2, S-/sqrt2, Sz], W_2 = [S-/sqrt2,
    S+/sqrt2, Sz]^T with unit S+- entries and Sz = diag(1, -1) (the values of
    P_1 printed there fix Sz this way).
    """
    sz = np.diag([1.0, -1.0])
    r2 = 1.0 / np.sqrt(2.0)
    W1 = np.zeros((2, 2, 1, 3))
    W1[:, :, 0, 0] = r2 * SP
    W1[:, :, 0, 1] = r2 * SM
    W1[:, :, 0, 2] = sz
    W2 = np.zeros((2, 2, 3, 1))
    W2[:, :, 0, 0] = r2 * SM
    W2[:, :, 1, 0] = r2 * SP
    W2[:, :, 2, 0] = sz
    t = [np.array([[0]]), np.array([[2], [-2], [0]]), np.array([[0]])]
    return MPO([W1, W2], SPIN_HALF_Q.copy(), t)


# ---- contraction of an MPO into a dense matrix -----------------------------

def mpo_to_dense(mpo):
    """Contract W_1 ... W_l over the MPO bonds into a (d^l, d^l) matrix (Sec. II)."""
    acc = mpo.W[0][:, :, 0, :]                       # (d, d, w1)
    acc = acc.reshape(acc.shape[0], acc.shape[1], -1)
    for Wi in mpo.W[1:]:
        # acc[(S), (T), b] * Wi[s, t, b, c] -> acc[(S s), (T t), c]
        n_out, n_in = acc.shape[0], acc.shape[1]
        acc = np.einsum("STb,stbc->SsTtc", acc, Wi)
        acc = acc.reshape(n_out * Wi.shape[0], n_in * Wi.shape[1], -1)
    return acc[:, :, 0]


# ---- dense Hamiltonians from Kronecker products ------------------------------

def _site_op(op, i, L, d):
    out = np.ones((1, 1))
    for k in range(L):
        out = np.kron(out, op if k == i else np.eye(d))
    return out


def _two_site_op(op_i, i, op_j, j, L, d):
    """op_i on site i times op_j on site j (i != j), as one Kronecker product."""
    out = np.ones((1, 1))
    for k in range(L):
        out = np.kron(out, op_i if k == i else (op_j if k == j else np.eye(d)))
    return out


def dense_spin_bonds(L, bonds, two_s=1):
    """Dense spin-S Hamiltonian sum Jxy (SxSx + SySy) + Jz SzSz over ``bonds``."""
    if two_s == 1:
        sp, sm, sz, d = SP, SM, SZ, 2
    else:
        sp, sm, sz, _, _ = spin_ops(two_s)
        d = two_s + 1
    sx = 0.5 * (sp + sm)
    sy_im = 0.5 * (sp - sm)          # S^y = -i * sy_im ; S^y S^y = -(sy_im x sy_im)
    H = np.zeros((d ** L, d ** L))
    for (i, j, jxy, jz) in bonds:
        H += jxy * _two_site_op(sx, i, sx, j, L, d)
        H -= jxy * _two_site_op(sy_im, i, sy_im, j, L, d)
        H += jz * _two_site_op(sz, i, sz, j, L, d)
    return H


def ring_bonds(L, J=1.0):
    """Heisenberg ring: nearest neighbours plus the link (0, L-1) closing it."""
    return [(i, i + 1, J, J) for i in range(L - 1)] + [(0, L - 1, J, J)]


def dense_xxz(L, J=1.0, Delta=1.0):
    return dense_spin_bonds(L, [(i, i + 1, J, J * Delta) for i in range(L - 1)])


def dense_hubbard(L, t_hop=1.0, U=0.0):
    """Dense Hubbard Hamiltonian on 2L fermionic modes via an explicit JW string."""
    nmodes = 2 * L

    def ann(k):
        out = np.ones((1, 1))
        for j in range(nmodes):
            out = np.kron(out, _PAR if j < k else (_ANN if j == k else I2))
        return out

    c = [ann(k) for k in range(nmodes)]
    dim = 2 ** nmodes
    H = np.zeros((dim, dim))
    for i in range(L - 1):
        for s in range(2):
            a, b = c[2 * i + s], c[2 * (i + 1) + s]
            H += -t_hop * (a.T @ b + b.T @ a)
    for i in range(L):
        H += U * (c[2 * i].T @ c[2 * i]) @ (c[2 * i + 1].T @ c[2 * i + 1])
    return H


def dense_charges(qphys, L):
    """Total charge of every basis state of L sites (first site most significant)."""
    q = np.zeros((1, qphys.shape[1]), dtype=np.int64)
    for _ in range(L):
        q = (q[:, None, :] + qphys[None, :, :]).reshape(-1, qphys.shape[1])
    return q
