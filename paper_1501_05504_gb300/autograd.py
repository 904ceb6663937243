"""Differentiable ground-state energy of a built-in model: E(theta) through DMRG3S.

The forward pass runs DMRG3S sweeps on the device (dmrg3s_sweep) for the
couplings theta (XXZ: (J, Delta); Hubbard: (t, U)) and returns the energy
<Psi|H|Psi>/<Psi|Psi> of the converged state.  The backward pass returns
dE/dtheta by Hellmann-Feynman, sum_i <G_i, dW_i/dtheta> / <Psi|Psi>, with the
MPO-entry gradients G_i (the energy network of Sec. II of arXiv:1501.05504
with W_i taken out; the environments on the far side of the orthogonality
centre are recomputed, not stored).  The library computes the energy and the
derivatives itself (dmrg3s_energy_grad): every MPO tensor of these models is
affine in each coupling, so it builds dW_i/dtheta_k = W_i(theta + e_k) -
W_i(theta) exactly.  This module only marshals the call.

The gradient is exact for the state that was found; it equals the derivative
of the ground-state energy to first order in the state's error.
"""
import numpy as np
import torch

from . import binding as b

_MODELS = {"xxz": b.MODEL_XXZ, "hubbard": b.MODEL_HUBBARD}


class GroundStateSolver:
    """DMRG3S ground states of one model at varying couplings.

    start: physical basis index of every site for the product start state
    (the Neel state [0, 1, 0, 1, ...] for XXZ, alternating up/down [2, 1, ...]
    for Hubbard).  warm: start from the previous solution's tensors (same
    gauge), which is what finite differences of the energy need.
    """

    def __init__(self, ctx, model, nsites, m_max, start, max_sweeps=16, conv_tol=1e-12,
                 alpha0=1e-2, lanczos_tol=1e-12, prec="fp64", warm=True):
        self.ctx = ctx
        self.model = _MODELS[model]
        self.nsites = int(nsites)
        self.m_max = int(m_max)
        self.start = list(start)
        self.max_sweeps = int(max_sweeps)
        self.conv_tol = float(conv_tol)
        self.alpha0 = float(alpha0)
        self.opts = b.update_opts(self.m_max, kmax=40, tol=lanczos_tol, prec=prec)
        self.warm = warm
        self._prev = None            # (site tensors, centre) of the last solution
        self.last_report = None

    def _mpo(self, params):
        return b.Mpo(self.model, self.nsites, tuple(float(x) for x in params)).sites()

    def _start_state(self, W):
        if self.warm and self._prev is not None:
            sites, centre = self._prev
            return b.dmrg3s_state_create(self.ctx, W, sites, None, None, centre)
        sites = b.product_state(W[0].qp, self.start)
        return b.dmrg3s_state_create(self.ctx, W, sites, None, None, self.nsites - 1)

    def solve(self, params):
        """(E, dE/dparams as a float64 numpy array) at the couplings `params`."""
        params = np.asarray(params, dtype=np.float64)
        W = self._mpo(params)
        st = self._start_state(W)
        try:
            self.last_report = b.dmrg3s_sweep(st, b.alpha_rule(self.alpha0), self.max_sweeps,
                                              self.conv_tol, self.opts)
            # the energy and the Hellmann-Feynman derivatives, from the MPO-entry
            # gradients and the model's dW/dtheta, all computed by the library
            energy, grad = b.dmrg3s_energy_grad(st, self.model, params)
            if self.warm:
                c, _ = st.centre()
                self._prev = ([st.site(i) for i in range(self.nsites)], c)
        finally:
            st.close()
        return energy, grad


class GroundStateEnergy(torch.autograd.Function):
    """E = GroundStateEnergy.apply(params, solver): differentiable in params."""

    @staticmethod
    def forward(ctx, params, solver):
        e, g = solver.solve(params.detach().cpu().numpy())
        ctx.save_for_backward(torch.as_tensor(g, dtype=params.dtype, device=params.device))
        return params.new_tensor(e)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


def ground_state_energy(params, solver):
    return GroundStateEnergy.apply(params, solver)
