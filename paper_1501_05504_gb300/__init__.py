"""GB300 (sm_103a) DMRG3S hot path: the effective-Hamiltonian application HA = L W A R,
the subspace-expansion term and the environment recursion of arXiv:1501.05504,
as hand-written CUDA kernels behind a C ABI (include/dmrg3s.h).

``binding`` is the thin ctypes layer over ``libdmrg3s.so``; build the library
with ``paper_1501_05504_gb300._build.build()`` (or ``__graft_entry__.build()``).
"""
from . import binding  # noqa: F401
from .binding import (  # noqa: F401
    Bond, Context, Env, MpoSite, Site, dmrg3s_apply_heff, dmrg3s_create, dmrg3s_destroy,
    dmrg3s_expand, dmrg3s_update_env, expanded_bond,
)
