"""GPU parity of the eigensolver, the DMRG3S local update and full sweeps.

The eigensolver value is unique (non-degenerate ground state of a random
symmetric H_eff); vectors are compared up to sign.  After a local update the
new basis is only defined up to a per-sector orthogonal rotation and sign,
so the comparison uses gauge-invariant quantities: lambda*, E_f, the
discarded weight, the kept dimension per charge sector and the two-site
wavefunction A~ B~ (up to a global sign).  Full sweeps are compared with the
oracle's converged energy and with exact diagonalisation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import seeded_inputs as si  # noqa: E402
from oracle import contract, dmrg3s as odm, exact, io, models  # noqa: E402
from parity import rel_err, site_to_dense  # noqa: E402


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05504_gb300 import binding
    binding.slib()
    return binding


@pytest.fixture(scope="module")
def ctx(b):
    c = b.dmrg3s_create(0, 1 << 30)
    yield c
    c.close()


def _window(kind, seed, m=48):
    """Two-site window: random symmetric boundary environments and MPO tensors."""
    rng = si.rng_for(seed)
    if kind == "dense":
        b0, b1, b2 = si.dense_bond(m), si.dense_bond(m + 3), si.dense_bond(m - 5)
        qp = np.zeros((2, 0), dtype=np.int64)
        t = np.zeros((5, 0), dtype=np.int64)
    elif kind == "u1":
        b0 = si.gaussian_bond(m, (1,), (2.5,), (2,), (4,))
        b1 = si.gaussian_bond(m + 4, (0,), (2.5,), (2,), (4,))
        b2 = si.gaussian_bond(m - 6, (1,), (2.5,), (2,), (4,))
        qp, t = si.XXZ_QP, si.XXZ_T
    elif kind == "u1u1_big":
        b0 = si._parity_filter(si.gaussian_bond(3 * m, (3, 1), (1.0, 1.0), (1, 2), (2, 2)), 3 * m)
        b1 = si._parity_filter(si.gaussian_bond(3 * m, (4, 0), (1.0, 1.0), (1, 2), (2, 2)), 3 * m)
        b2 = si._parity_filter(si.gaussian_bond(2 * m, (5, 1), (1.0, 1.0), (1, 2), (2, 2)), 2 * m)
        qp, t = si.HUB_QP, si.HUB_T
    else:
        b0 = si._parity_filter(si.gaussian_bond(m, (3, 1), (1.5, 1.5), (1, 2), (3, 3)), m)
        b1 = si._parity_filter(si.gaussian_bond(m + 4, (4, 0), (1.5, 1.5), (1, 2), (3, 3)), m + 4)
        b2 = si._parity_filter(si.gaussian_bond(m - 6, (5, 1), (1.5, 1.5), (1, 2), (3, 3)), m - 6)
        qp, t = si.HUB_QP, si.HUB_T
    Le = si.symmetric_env(rng, t, b0)
    Re = si.symmetric_env(rng, t, b2)
    W0 = si.symmetric_mpo_site(rng, qp, t, t)
    W1 = si.symmetric_mpo_site(rng, qp, t, t)
    M0 = si.random_site(rng, qp, b0, b1)
    M1 = si.random_site(rng, qp, b1, b2)
    return dict(L=Le, R=Re, W=[W0, W1], M=[M0, M1], qp=qp, t=t)


# Truncation cutoff of the parity tests: above the eigensolver's noise floor
# (its 1e-12 residual leaves singular values up to ~1e-10 s_max that are not
# part of the solution), so both sides keep the same states.
EPS = 1e-9


def _oracle_window(w, centre, m_max, alpha):
    mpo = models.MPO([w["W"][0]["W"], w["W"][1]["W"]], w["qp"], [w["t"], w["t"], w["t"]])
    Ms, qs = [], []
    for k, M in enumerate(w["M"]):
        D, ql, qr = io.site_dense(M)
        Ms.append(D)
        if k == 0:
            qs.append(ql)
        qs.append(qr)
    mps = odm.MPS(Ms, qs, w["qp"])
    o = odm.SweepOptions(m_max=m_max, trunc_eps=EPS, lanczos_kmax=80, lanczos_tol=1e-12)
    o.alpha = odm.AlphaRule(alpha0=alpha, fixed=True)
    return odm.DMRG3S(mpo, mps, o, left_env=io.env_dense(w["L"]), right_env=io.env_dense(w["R"]),
                      centre=centre)


def _gpu_window(b, ctx, w, centre):
    W = [b.mpo_from_neutral(x) for x in w["W"]]
    M = [b.site_from_neutral(x) for x in w["M"]]
    return b.dmrg3s_state_create(ctx, W, M, b.env_from_neutral(w["L"]), b.env_from_neutral(w["R"]),
                                 centre)


def _sector_dims(bond):
    return sorted((tuple(int(v) for v in q), int(d)) for q, d in zip(bond.q, bond.dim))


def _oracle_sector_dims(q):
    out = {}
    for row in q:
        k = tuple(int(v) for v in row)
        out[k] = out.get(k, 0) + 1
    return sorted(out.items())


@pytest.mark.parametrize("kind,seed", [("dense", 1), ("u1", 2), ("u1u1", 3)])
def test_eigensolve_matches_oracle(b, ctx, kind, seed):
    w = _window(kind, seed)
    # a one-site problem: L on M0.left, a symmetric random R on M0.right
    R1 = si.symmetric_env(si.rng_for(seed + 100), w["t"], w["M"][0]["right"])
    gL, gR1 = b.env_from_neutral(w["L"]), b.env_from_neutral(R1)
    gW = b.mpo_from_neutral(w["W"][0])
    gM = b.site_from_neutral(w["M"][0])
    lam, it = b.dmrg3s_eigensolve(ctx, gL, gW, gR1, gM, kmax=80, tol=1e-12)
    Ld, Rd, Md = io.env_dense(w["L"]), io.env_dense(R1), io.site_dense(w["M"][0])[0]
    lam_o, x_o, it_o = odm.lanczos_ground(lambda v: contract.apply_heff(Ld, w["W"][0]["W"], Rd, v), Md,
                                          kmax=80, tol=1e-12)
    assert abs(lam - lam_o) < 1e-10 * max(1.0, abs(lam_o))
    x_p = site_to_dense(b, gM)
    assert abs(abs(np.vdot(x_p, x_o)) - 1.0) < 1e-8


def _heff_gap(orc, direction):
    """lambda_2 - lambda_1 of the centre site's H_eff (scipy Lanczos on the oracle's product)."""
    import scipy.sparse.linalg as sla
    i = 0 if direction == 1 else 1
    Le, Re, W = orc.Lenv[i], orc.Renv[i], orc.mpo.W[i]
    shape = orc.mps.M[i].shape
    n = int(np.prod(shape))
    op = sla.LinearOperator((n, n), dtype=np.float64,
                            matvec=lambda v: contract.apply_heff(Le, W, Re, v.reshape(shape)).reshape(-1))
    vals = np.sort(sla.eigsh(op, k=2, which="SA", tol=1e-12, v0=orc.mps.M[i].reshape(-1),
                             return_eigenvectors=False))
    return max(vals[1] - vals[0], 1e-300)


def _cut_gap(orc, direction, alpha, m_max):
    """Relative gap s_k - s_{k+1} of the expanded tensor's spectrum at the cut k = m_max."""
    i = 0 if direction == 1 else 1
    Le, Re, W = orc.Lenv[i], orc.Renv[i], orc.mpo.W[i]
    lam, Ms, _ = odm.lanczos_ground(lambda v: contract.apply_heff(Le, W, Re, v), orc.mps.M[i],
                                    kmax=80, tol=1e-12)
    if direction == 1:
        Mt = np.concatenate([Ms, contract.expansion_term_lr(Le, W, Ms, alpha)], axis=2)
        X = Mt.reshape(-1, Mt.shape[2])
    else:
        Mt = np.concatenate([Ms, contract.expansion_term_rl(Re, W, Ms, alpha)], axis=1)
        X = np.transpose(Mt, (1, 0, 2)).reshape(Mt.shape[1], -1)
    s = np.linalg.svd(X, compute_uv=False)
    k = min(m_max, int(np.sum(s > EPS * s[0])))
    if k >= len(s):
        return 1.0
    return (s[k - 1] - s[k]) / s[0]


@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("kind,seed", [("dense", 11), ("u1", 12), ("u1u1", 13), ("u1u1_big", 14)])
@pytest.mark.parametrize("m_max", [40, 100000])
@pytest.mark.parametrize("svd", ["jacobi", "gesvd"])
def test_local_update_matches_oracle(b, ctx, kind, seed, direction, m_max, svd):
    """m_max = 100000 keeps every state (no truncation): the state must be reproduced
    exactly.  m_max = 40 truncates: the kept subspace is then defined only up to
    the first-order perturbation eps / gap of the spectrum at the cut, and the
    two-site state is compared within 1e-9 / gap."""
    w = _window(kind, seed)
    centre = 0 if direction == 1 else 1
    alpha = 0.15
    orc = _oracle_window(w, centre, m_max, alpha)
    gap = _cut_gap(orc, direction, alpha, m_max)
    gap_h = _heff_gap(orc, direction)
    lam_o, ef_o = orc.update_lr(0) if direction == 1 else orc.update_rl(1)
    st = _gpu_window(b, ctx, w, centre)
    info = b.dmrg3s_local_update(st, direction, alpha, b.update_opts(m_max, kmax=80, tol=1e-12,
                                                                     eps=EPS, svd=svd))
    assert abs(info["lambda"] - lam_o) < 1e-9 * max(1.0, abs(lam_o))
    assert abs(info["energy_after"] - ef_o) < 1e-8 * max(1.0, abs(ef_o))
    g0, g1 = st.site(0), st.site(1)
    assert _sector_dims(g0.right) == _oracle_sector_dims(orc.mps.q[1])
    psi_p = np.einsum("sxa,tay->sxty", site_to_dense(b, g0), site_to_dense(b, g1))
    psi_o = np.einsum("sxa,tay->sxty", orc.mps.M[0], orc.mps.M[1])
    err = min(rel_err(psi_p, psi_o), rel_err(-psi_p, psi_o))
    # both eigenvectors satisfy |H x - lambda x| <= tol |lambda|, so each is
    # within tol |lambda| / gap_H of the exact one (gap_H: lowest two eigenvalues)
    assert err < min(1e-3, 4e-12 * max(1.0, abs(lam_o)) / gap_h + 1e-9 / gap)
    # the new centre-side tensor is orthonormal (A~ left-, B~ right-normalised)
    T = site_to_dense(b, g0 if direction == 1 else g1)
    G = np.einsum("sxa,sxb->ab", T, T) if direction == 1 else np.einsum("sax,sbx->ab", T, T)
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-12
    st.close()


def _neel_state(b, ctx, mpo_sites, L):
    spec = si.product_state_sites(si.XXZ_QP, [0, 1] * (L // 2))
    M = [b.site_from_neutral(x) for x in spec]
    return b.dmrg3s_state_create(ctx, mpo_sites, M, None, None, L - 1)


def test_sweep_u1_heisenberg_reaches_ed(b, ctx):
    L = 10
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 1.0)).sites()
    st = _neel_state(b, ctx, W, L)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 8, 1e-9, b.update_opts(32))
    e0 = exact.ed_ground_energy(models.dense_xxz(L, 1.0, 1.0),
                                models.dense_charges(models.SPIN_HALF_Q, L), [0])
    assert rep["converged"]
    assert abs(rep["energy"] - e0) < 1e-10 * abs(e0)
    # the oracle on the same start reaches the same energy
    mpo = models.mpo_xxz(L, 1.0, 1.0)
    olog = odm.DMRG3S(mpo, odm.product_state(mpo.qphys, [0, 1] * (L // 2)),
                      odm.SweepOptions(m_max=32, max_sweeps=8)).run()
    assert abs(rep["energy"] - olog.energies[-1]) < 1e-10 * abs(e0)
    st.close()


def test_sweep_alpha_zero_stays_stuck(b, ctx):
    L = 10
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 1.0)).sites()
    st = _neel_state(b, ctx, W, L)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(0.0, fixed=True), 2, 1e-9, b.update_opts(32))
    assert abs(rep["energy"] - (-(L - 1) / 4.0)) < 1e-12
    st.close()


def test_sweep_hubbard_matches_ed(b, ctx):
    L, U = 4, 8.0
    W = b.Mpo(b.MODEL_HUBBARD, L, (1.0, U)).sites()
    spec = si.product_state_sites(si.HUB_QP, [2, 1] * (L // 2))
    st = b.dmrg3s_state_create(ctx, W, [b.site_from_neutral(x) for x in spec], None, None, L - 1)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 10, 1e-10, b.update_opts(64))
    e0 = exact.ed_ground_energy(models.dense_hubbard(L, 1.0, U), models.dense_charges(models.HUB_Q, L),
                                [L, 0])
    assert abs(rep["energy"] - e0) < 1e-9 * abs(e0)
    st.close()


def test_sweep_dense_random_start(b, ctx):
    """No symmetry, random start (left-normalised on the device by gauge moves)."""
    L, m = 10, 32
    W = b.Mpo(b.MODEL_XXZ, L, (1.0, 1.0)).sites()
    for s in W:     # the dense problem drops the charges
        s.qp = np.zeros((2, 0), np.int32)
        s.tl = np.zeros((s.tl.shape[0], 0), np.int32)
        s.tr = np.zeros((s.tr.shape[0], 0), np.int32)
    Ms = si.random_dense_mps(si.rng_for(1001), L, 2, m)
    st = b.dmrg3s_state_create(ctx, W, [b.site_from_neutral(x) for x in si.dense_mps_sites(Ms)],
                               None, None, 0)
    gauge = b.update_opts(10 ** 6, skip_eigensolver=True)
    for _ in range(L - 1):
        b.dmrg3s_local_update(st, 1, 0.0, gauge)
    rep = b.dmrg3s_sweep(st, b.alpha_rule(1e-2), 8, 1e-10, b.update_opts(m))
    e0 = exact.ed_ground_energy(models.dense_xxz(L, 1.0, 1.0))
    assert abs(rep["energy"] - e0) < 1e-10 * abs(e0)
    st.close()
