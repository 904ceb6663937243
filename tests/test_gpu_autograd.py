"""dE/d(couplings) through torch.autograd on the DMRG3S ground state.

Pins: the homogeneity identity J dE/dJ = E of the XXZ chain at fixed Delta,
Hellmann-Feynman derivatives <psi|dH/dtheta|psi> of the exact ground state
from exact diagonalisation (the oracle's ED and Hamiltonian builders), and
central finite differences of the converged energy (h = 1e-4, warm-started
same-gauge runs), within the gradient tolerance 1e-6 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import exact, models  # noqa: E402


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


def _ed_hellmann_feynman(H, dHs, charges, sector):
    """Ground energy and <psi|dH|psi> of the exact ground state in a charge sector."""
    idx = np.nonzero(np.all(charges == np.asarray(sector)[None, :], axis=1))[0]
    h = H[np.ix_(idx, idx)]
    w, v = np.linalg.eigh(h)
    psi = v[:, 0]
    return w[0], [float(psi @ dH[np.ix_(idx, idx)] @ psi) for dH in dHs]


def test_xxz_energy_gradient(b, ctx):
    from paper_1501_05504_gb300.autograd import GroundStateSolver, ground_state_energy
    L, J, delta = 12, 1.0, 0.7
    solver = GroundStateSolver(ctx, "xxz", L, 64, [0, 1] * (L // 2))
    theta = torch.tensor([J, delta], dtype=torch.float64, requires_grad=True)
    E = ground_state_energy(theta, solver)
    E.backward()
    g = theta.grad.numpy()
    # exact diagonalisation in the S^z = 0 sector
    q = models.dense_charges(models.SPIN_HALF_Q, L)
    H = models.dense_xxz(L, J, delta)
    dJ = models.dense_xxz(L, 1.0, delta)                     # H is linear in J at fixed Delta
    dD = models.dense_xxz(L, J, 1.0) - models.dense_xxz(L, J, 0.0)
    e0, (gJ, gD) = _ed_hellmann_feynman(H, [dJ, dD], q, [0])
    assert abs(E.item() - e0) < 1e-9 * abs(e0)
    assert abs(J * g[0] - E.item()) < 1e-10 * abs(E.item())
    assert abs(g[0] - gJ) < 1e-6 * abs(gJ)
    assert abs(g[1] - gD) < 1e-6 * abs(gD)
    # central finite difference in Delta from the converged state
    h = 1e-4
    ep, _ = solver.solve([J, delta + h])
    em, _ = solver.solve([J, delta - h])
    fd = (ep - em) / (2 * h)
    assert abs(fd - g[1]) < 1e-6 * abs(g[1])


def test_hubbard_energy_gradient(b, ctx):
    from paper_1501_05504_gb300.autograd import GroundStateSolver, ground_state_energy
    L, t, U = 6, 1.0, 8.0
    solver = GroundStateSolver(ctx, "hubbard", L, 64, [2, 1] * (L // 2))
    theta = torch.tensor([t, U], dtype=torch.float64, requires_grad=True)
    E = ground_state_energy(theta, solver)
    E.backward()
    g = theta.grad.numpy()
    q = models.dense_charges(models.HUB_Q, L)
    H = models.dense_hubbard(L, t, U)
    dt = models.dense_hubbard(L, 1.0, U) - models.dense_hubbard(L, 0.0, U)
    dU = models.dense_hubbard(L, t, 1.0) - models.dense_hubbard(L, t, 0.0)
    e0, (gt, gU) = _ed_hellmann_feynman(H, [dt, dU], q, [L, 0])
    assert abs(E.item() - e0) < 1e-9 * abs(e0)
    # E is homogeneous of degree one in (t, U)
    assert abs(t * g[0] + U * g[1] - E.item()) < 1e-9 * abs(E.item())
    assert abs(g[0] - gt) < 1e-6 * abs(gt)
    assert abs(g[1] - gU) < 1e-6 * abs(gU)
    h = 1e-4
    ep, _ = solver.solve([t, U + h])
    em, _ = solver.solve([t, U - h])
    assert abs((ep - em) / (2 * h) - g[1]) < 1e-6 * abs(g[1]) + 1e-8
