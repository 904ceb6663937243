"""Pins of the oracle's contractions (CPU only).

* H_eff applied by (((L M) W) R) equals the dense Hamiltonian (built from
  Kronecker products, not from the MPO) projected onto the MPS basis of the
  centre site: (l_{i-1} x 1 x r_{i+1})^T H (l_{i-1} x 1 x r_{i+1})  (Sec. II, Sec. V);
* <Psi|H|Psi> from the environments equals the dense expectation value at
  every split point (Sec. II);
* the two-spin example of Sec. IV C reproduces the printed matrices;
* subspace expansion leaves the state unchanged (Sec. IV A) and the SVD
  restores orthonormality; truncation error equals the discarded weight;
* the MPO-entry gradient equals the exact derivative of <H>(Delta).
"""
import json
import os

import numpy as np
import pytest

import seeded_inputs as si
from oracle import contract, dmrg3s, io, labels, models

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- helpers (test side) ---------------------------------------------------------

def _left_basis(As):
    l = np.ones((1, 1))
    for A in As:
        l = np.einsum("Pa,sab->Psb", l, A).reshape(-1, A.shape[2])
    return l


def _right_basis(Bs):
    r = np.ones((1, 1))
    for B in reversed(Bs):
        r = np.einsum("sab,bR->asR", B, r).reshape(B.shape[1], -1)
    return r


def _mixed_canonical(L, d, m, centre, seed):
    rng = np.random.default_rng(seed)
    Ms = si.random_dense_mps(rng, L, d, m)
    As = dmrg3s.left_normalise(Ms)
    Bs = dmrg3s.right_normalise(Ms)
    return As[:centre], rng.standard_normal(Ms[centre].shape), Bs[centre + 1:]


def _env_chain(mpo, As, Bs):
    Le = np.ones((1, 1, 1))
    for i, A in enumerate(As):
        Le = contract.left_env(Le, mpo.W[i], A)
    Re = np.ones((1, 1, 1))
    for k, B in enumerate(reversed(Bs)):
        i = mpo.L - 1 - k
        Re = contract.right_env(Re, mpo.W[i], B)
    return Le, Re


def heff_projection_error(apply, mpo, H, As, x, Bs):
    """max |apply(L, W, R, x) - Phi^T H Phi x| for the basis map Phi of the centre site."""
    centre = len(As)
    Le, Re = _env_chain(mpo, As, Bs)
    l, r = _left_basis(As), _right_basis(Bs)
    d = x.shape[0]
    Phi = np.einsum("Pa,st,bR->PsRtab", l, np.eye(d), r).reshape(H.shape[0], -1)
    ref = (Phi.T @ (H @ (Phi @ x.reshape(-1)))).reshape(x.shape)
    got = apply(Le, mpo.W[centre], Re, x)
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


# ---- H_eff ---------------------------------------------------------------------------

@pytest.mark.parametrize("centre", [0, 2, 5])
def test_heff_equals_projected_hamiltonian_xxz(centre):
    L = 6
    mpo = models.mpo_xxz(L, 1.0, 0.6)
    H = models.dense_xxz(L, 1.0, 0.6)
    As, x, Bs = _mixed_canonical(L, 2, 8, centre, seed=centre)
    assert heff_projection_error(contract.apply_heff, mpo, H, As, x, Bs) < 1e-13


@pytest.mark.parametrize("centre", [0, 1, 3])
def test_heff_equals_projected_hamiltonian_hubbard(centre):
    L = 4
    mpo = models.mpo_hubbard(L, 1.0, 3.0)
    H = models.dense_hubbard(L, 1.0, 3.0)
    As, x, Bs = _mixed_canonical(L, 4, 16, centre, seed=10 + centre)
    assert heff_projection_error(contract.apply_heff, mpo, H, As, x, Bs) < 1e-13


def test_heff_ordered_equals_unordered_sum():
    rng = np.random.default_rng(3)
    L_ = rng.standard_normal((3, 5, 4))
    R_ = rng.standard_normal((2, 6, 7))
    W = rng.standard_normal((2, 2, 3, 2))
    M = rng.standard_normal((2, 4, 7))
    a = contract.apply_heff(L_, W, R_, M)
    b = contract.apply_heff_literal(L_, W, R_, M)
    assert np.abs(a - b).max() < 1e-12


def _u1_problem(seed, m=24):
    rng = si.rng_for(seed)
    left = si.gaussian_bond(m, (1,), (2.0,), (2,), (3,))
    right = si.gaussian_bond(m, (0,), (2.0,), (2,), (3,))
    Le = si.symmetric_env(rng, si.XXZ_T, left, identity_channels=(4,))
    Re = si.symmetric_env(rng, si.XXZ_T, right, identity_channels=(0,))
    mpo = models.mpo_xxz(6, 1.0, 0.8)
    return mpo.W[2], io.env_dense(Le), io.env_dense(Re), left, right


def test_heff_rows_equal_the_rows_of_the_unordered_sum():
    """The row-restricted H_eff equals the matching rows of the literal sum."""
    rng = np.random.default_rng(7)
    d, wl, wr, ml, mr = 3, 4, 5, 6, 7
    L = rng.standard_normal((wl, ml, ml))
    W = rng.standard_normal((d, d, wl, wr))
    R = rng.standard_normal((wr, mr, mr))
    M = rng.standard_normal((d, ml, mr))
    rows = [5, 0, 3]
    full = contract.apply_heff_literal(L, W, R, M)
    assert np.abs(contract.apply_heff_rows(L, W, R, M, rows) - full[:, rows, :]).max() < 1e-12


def test_heff_symmetric_on_symmetric_environments():
    W, Le, Re, left, right = _u1_problem(7)
    rng = np.random.default_rng(8)
    x = io.site_dense(si.random_site(rng, si.XXZ_QP, left, right))[0]
    y = io.site_dense(si.random_site(rng, si.XXZ_QP, left, right))[0]
    a = np.vdot(x, contract.apply_heff(Le, W, Re, y))
    b = np.vdot(contract.apply_heff(Le, W, Re, x), y)
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))


def test_heff_preserves_charge_structure():
    W, Le, Re, left, right = _u1_problem(9)
    rng = np.random.default_rng(10)
    x, ql, qr = io.site_dense(si.random_site(rng, si.XXZ_QP, left, right))
    mask = labels.site_mask(si.XXZ_QP, ql, qr)
    y = contract.apply_heff(Le, W, Re, x)
    assert np.all(y[~mask] == 0.0)


# ---- energy from environments ----------------------------------------------------------

def test_energy_identical_from_every_split():
    L = 6
    mpo = models.mpo_xxz(L, 1.0, 1.3)
    H = models.dense_xxz(L, 1.0, 1.3)
    rng = np.random.default_rng(5)
    Ms = dmrg3s.left_normalise(si.random_dense_mps(rng, L, 2, 8))
    mps = dmrg3s.MPS(Ms, [None] * (L + 1), np.zeros((2, 0), dtype=np.int64))
    psi = dmrg3s.mps_to_dense(mps)
    e_ref = float(psi @ H @ psi) / float(psi @ psi)
    # move the centre from the right end to the left by SVD, checking every split
    Ms = list(Ms)
    for c in range(L - 1, -1, -1):
        Le, Re = _env_chain(mpo, Ms[:c], Ms[c + 1:])
        e = contract.rayleigh(Le, mpo.W[c], Re, Ms[c])
        assert abs(e - e_ref) < 1e-12 * abs(e_ref)
        if c > 0:
            B, US, _ = dmrg3s.truncate_rl(Ms[c], np.zeros((2, 0), dtype=np.int64),
                                          np.zeros((Ms[c].shape[1], 0), dtype=np.int64),
                                          np.zeros((Ms[c].shape[2], 0), dtype=np.int64), 10 ** 6)
            Ms[c] = B
            Ms[c - 1] = np.einsum("sxy,yk->sxk", Ms[c - 1], US)


# ---- the two-spin example (Sec. IV C) ------------------------------------------------------

def _golden_two_spin():
    with open(os.path.join(GOLDEN, "two_spin_example.json")) as f:
        return json.load(f)


def _ev(expr, a, b):
    return float(eval(expr, {"sqrt": np.sqrt, "a": a, "b": b}))


def two_spin_errors(expansion_lr, a, b):
    g = _golden_two_spin()
    mpo = models.mpo_two_spin_example()
    A1 = np.array([[[a]], [[np.sqrt(1 - a * a)]]])
    B2 = np.array([[[b]], [[np.sqrt(1 - b * b)]]])
    L0 = np.ones((1, 1, 1))
    P = expansion_lr(L0, mpo.W[0], A1, 1.0)
    errs = {}
    errs["P1"] = max(abs(P[0, 0, k] - _ev(e, a, b)) for k, e in enumerate(g["P1"]["up"]))
    errs["P1"] = max(errs["P1"], max(abs(P[1, 0, k] - _ev(e, a, b)) for k, e in enumerate(g["P1"]["down"])))
    At = np.concatenate([A1, P], axis=2)
    Bt = np.concatenate([B2, np.zeros((2, 3, 1))], axis=1)
    errs["A1p"] = max(max(abs(At[0, 0, k] - _ev(e, a, b)) for k, e in enumerate(g["A1_prime"]["up"])),
                      max(abs(At[1, 0, k] - _ev(e, a, b)) for k, e in enumerate(g["A1_prime"]["down"])))
    errs["B2p"] = max(max(abs(Bt[0, k, 0] - _ev(e, a, b)) for k, e in enumerate(g["B2_prime"]["up"])),
                      max(abs(Bt[1, k, 0] - _ev(e, a, b)) for k, e in enumerate(g["B2_prime"]["down"])))
    nosym = np.zeros((2, 0), dtype=np.int64)
    A2, SV, _ = dmrg3s.truncate_lr(At, nosym, np.zeros((1, 0), dtype=np.int64),
                                   np.zeros((4, 0), dtype=np.int64), 2)
    # A'' is the identity up to the order and signs of the new basis states (the
    # order of the singular values depends on a): align by the row of A'' that is hit.
    perm = [int(np.argmax(np.abs(A2[s, 0, :]))) for s in range(2)]
    sign = [float(np.sign(A2[s, 0, perm[s]])) for s in range(2)]
    A2n = np.stack([A2[:, 0, perm[s]] * sign[s] for s in range(2)], axis=1)
    SVn = np.stack([SV[perm[s], :] * sign[s] for s in range(2)], axis=0)
    errs["A1pp"] = np.abs(A2n - np.array([[_ev(e, a, b) for e in g["A1_second"]["up"]],
                                          [_ev(e, a, b) for e in g["A1_second"]["down"]]])).max()
    errs["SV"] = np.abs(SVn - np.array([[_ev(e, a, b) for e in row] for row in g["SVdag"]])).max()
    B2pp = np.einsum("kx,sxy->sky", SVn, Bt)
    errs["B2pp"] = max(max(abs(B2pp[0, k, 0] - _ev(e, a, b)) for k, e in enumerate(g["B2_second"]["up"])),
                       max(abs(B2pp[1, k, 0] - _ev(e, a, b)) for k, e in enumerate(g["B2_second"]["down"])))
    psi0 = np.einsum("sxa,tay->st", A1, B2)
    psi1 = np.einsum("sxa,tay->st", A2, np.einsum("kx,sxy->sky", SV, Bt))
    errs["state"] = np.abs(psi0 - psi1).max()
    return errs


@pytest.mark.parametrize("a,b", [(0.3, 0.6), (0.8, 0.1), (0.55, 0.9)])
def test_two_spin_example_printed_values(a, b):
    errs = two_spin_errors(contract.expansion_term_lr, a, b)
    for k, v in errs.items():
        assert v < 1e-14, (k, v)


# ---- expansion, truncation, orthonormality -------------------------------------------------

def _warm_u1_state(L=8, m=16, sweeps=1):
    mpo = models.mpo_xxz(L, 1.0, 1.0)
    mps = dmrg3s.product_state(mpo.qphys, [0, 1] * (L // 2))
    drv = dmrg3s.DMRG3S(mpo, mps, dmrg3s.SweepOptions(m_max=m, max_sweeps=sweeps))
    drv.run()
    return mpo, drv


def expansion_lr_errors(expand):
    """Deviations of the state and of the gauge after expansion (with ``expand``) + SVD."""
    mpo, drv = _warm_u1_state()
    mps, i = drv.mps, 3
    psi_before = dmrg3s.mps_to_dense(mps)
    M, Mn = mps.M[i], mps.M[i + 1]
    P = expand(drv.Lenv[i], mpo.W[i], M, 0.37)
    Mt = np.concatenate([M, P], axis=2)
    Bt = np.concatenate([Mn, np.zeros((Mn.shape[0], P.shape[2], Mn.shape[2]))], axis=1)
    mps2 = dmrg3s.MPS(list(mps.M), list(mps.q), mps.qphys)
    mps2.M[i], mps2.M[i + 1] = Mt, Bt
    errs = {"expanded": np.abs(dmrg3s.mps_to_dense(mps2) - psi_before).max()}
    qr_t = np.concatenate([mps.q[i + 1], labels.combine(mpo.t[i + 1], mps.q[i + 1])], axis=0)
    A, SV, qn = dmrg3s.truncate_lr(Mt, mps.qphys, mps.q[i], qr_t, 10 ** 6)
    errs["gauge"] = np.abs(np.einsum("sxa,sxb->ab", A, A) - np.eye(A.shape[2])).max()
    errs["charges"] = float(np.abs(A[~labels.site_mask(mps.qphys, mps.q[i], qn)]).max(initial=0.0))
    mps2.M[i], mps2.M[i + 1] = A, np.einsum("kx,sxy->sky", SV, Bt)
    errs["after_svd"] = np.abs(dmrg3s.mps_to_dense(mps2) - psi_before).max()
    # the expanded basis must also carry the expansion term: its weight survives the SVD
    errs["p_kept"] = abs(np.linalg.norm(A.reshape(-1, A.shape[2]) @ SV) - np.linalg.norm(Mt))
    return errs


def test_expansion_lr_leaves_state_unchanged_and_svd_restores_gauge():
    errs = expansion_lr_errors(contract.expansion_term_lr)
    assert errs["expanded"] < 1e-15
    assert errs["gauge"] < 1e-13
    assert errs["charges"] == 0.0
    assert errs["after_svd"] < 1e-13
    assert errs["p_kept"] < 1e-12


def test_expansion_rl_leaves_state_unchanged():
    mpo, drv = _warm_u1_state()
    mps = drv.mps
    # after run() the centre is at the right end; do a right-to-left step by hand at site L-1
    i = mps.L - 1
    psi_before = dmrg3s.mps_to_dense(mps)
    M, Mp = mps.M[i], mps.M[i - 1]
    P = contract.expansion_term_rl(drv.Renv[i], mpo.W[i], M, 0.21)
    Mt = np.concatenate([M, P], axis=1)
    At = np.concatenate([Mp, np.zeros((Mp.shape[0], Mp.shape[1], P.shape[1]))], axis=2)
    mps2 = dmrg3s.MPS(list(mps.M), list(mps.q), mps.qphys)
    mps2.M[i], mps2.M[i - 1] = Mt, At
    assert np.abs(dmrg3s.mps_to_dense(mps2) - psi_before).max() < 1e-15
    ql_t = np.concatenate([mps.q[i], labels.combine(mpo.t[i], mps.q[i])], axis=0)
    B, US, qn = dmrg3s.truncate_rl(Mt, mps.qphys, ql_t, mps.q[i + 1], 10 ** 6)
    assert np.abs(np.einsum("sax,sbx->ab", B, B) - np.eye(B.shape[1])).max() < 1e-13
    mps2.M[i], mps2.M[i - 1] = B, np.einsum("sxy,yk->sxk", At, US)
    assert np.abs(dmrg3s.mps_to_dense(mps2) - psi_before).max() < 1e-13


def expansion_rl_mirror_error(expand_rl, seed=7):
    """Largest deviation of the right-to-left expansion term from the mirror
    image of the left-to-right one (Sec. IV B).

    Reflecting the chain swaps the two MPS bonds of M, the two MPO bonds of W
    and the roles of L and R.  The R->L term on the chain is then the L->R
    term on the reflected chain with its two bond indices exchanged:
      P_rl[s', (bl, al), ar'] = P_lr^mirror[s', ar', (bl, al)],
      P_lr^mirror = expansion_term_lr(R, W with (bl, br) swapped, M with (al, ar) swapped).
    The L->R term is pinned by the printed two-spin example (Sec. IV C).
    Checked on random unsymmetric tensors of unequal bond dimensions (so a
    transposed operand or a swapped index cannot cancel) and on the XXZ MPO
    of a warm U(1) state."""
    rng = np.random.default_rng(seed)
    cases = []
    d, wl, wr, ml, mr = 3, 4, 5, 6, 7
    cases.append((rng.standard_normal((wr, mr, mr)), rng.standard_normal((d, d, wl, wr)),
                  rng.standard_normal((d, ml, mr))))
    mpo, drv = _warm_u1_state()
    i = mpo.L - 2      # the right environment of site L-2, built from the last site
    Re = contract.right_env(drv.Renv[i + 1], mpo.W[i + 1], drv.mps.M[i + 1])
    cases.append((Re, mpo.W[i], drv.mps.M[i]))
    err = 0.0
    for R, W, M in cases:
        got = expand_rl(R, W, M, 0.43)
        mirror = contract.expansion_term_lr(R, np.transpose(W, (0, 1, 3, 2)),
                                            np.transpose(M, (0, 2, 1)), 0.43)
        ref = np.transpose(mirror, (0, 2, 1))
        if got.shape != ref.shape:
            return np.inf
        err = max(err, float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)))
    return err


def test_expansion_rl_is_the_mirror_of_expansion_lr():
    assert expansion_rl_mirror_error(contract.expansion_term_rl) < 1e-14


def test_expansion_rl_basis_carries_the_expansion_term():
    """After [M; P] and the SVD the kept right basis still holds all of M~ (no
    truncation), P included (the mirror of the L->R check)."""
    mpo, drv = _warm_u1_state()
    mps = drv.mps
    i = mps.L - 1
    M = mps.M[i]
    P = contract.expansion_term_rl(drv.Renv[i], mpo.W[i], M, 0.29)
    assert np.linalg.norm(P) > 1e-3 * np.linalg.norm(M)
    Mt = np.concatenate([M, P], axis=1)
    ql_t = np.concatenate([mps.q[i], labels.combine(mpo.t[i], mps.q[i])], axis=0)
    B, US, _ = dmrg3s.truncate_rl(Mt, mps.qphys, ql_t, mps.q[i + 1], 10 ** 6)
    rebuilt = np.einsum("yk,skx->syx", US, B)
    assert np.abs(rebuilt - Mt).max() < 1e-13 * np.abs(Mt).max()


def test_truncation_error_is_discarded_weight():
    rng = np.random.default_rng(4)
    nos = np.zeros((2, 0), dtype=np.int64)
    Mt = rng.standard_normal((2, 6, 15))
    A, SV, _ = dmrg3s.truncate_lr(Mt, nos, np.zeros((6, 0), dtype=np.int64),
                                  np.zeros((15, 0), dtype=np.int64), 4)
    s = np.linalg.svd(Mt.reshape(12, 15), compute_uv=False)
    err = np.linalg.norm(Mt.reshape(12, 15) - A.reshape(12, 4) @ SV) ** 2
    assert abs(err - np.sum(s[4:] ** 2)) < 1e-12 * np.sum(s ** 2)


# ---- gradients ---------------------------------------------------------------------

def test_mpo_gradient_equals_exact_derivative():
    L, J, D = 6, 1.0, 0.7
    rng = np.random.default_rng(12)
    Ms = si.random_dense_mps(rng, L, 2, 8)
    mps = dmrg3s.MPS(Ms, [None] * (L + 1), np.zeros((2, 0), dtype=np.int64))
    psi = dmrg3s.mps_to_dense(mps)
    nrm = float(psi @ psi)
    # d<H>/dDelta exactly: <H> is linear in Delta, so a unit difference is the derivative
    dE = (float(psi @ models.dense_xxz(L, J, D + 1.0) @ psi) - float(psi @ models.dense_xxz(L, J, D) @ psi)) / nrm
    mpo = models.mpo_xxz(L, J, D)
    dW = [a - b for a, b in zip(models.mpo_xxz(L, J, D + 1.0).W, mpo.W)]
    tot = 0.0
    for i in range(L):
        Le, Re = _env_chain(mpo, Ms[:i], Ms[i + 1:])
        G = contract.mpo_gradient(Le, Re, Ms[i])
        tot += float(np.sum(G * dW[i]))
    assert abs(tot / nrm - dE) < 1e-12 * max(1.0, abs(dE))
