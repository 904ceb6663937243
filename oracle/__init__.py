"""FP64 CPU oracle for DMRG3S (Hubig, McCulloch, Schollwoeck, Wolf, arXiv:1501.05504).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test-suite, the smoke check of the package
entry point and the CPU-baseline leg of the benchmark use it.  It shares no
code with the CUDA path; the only inputs the two have in common come from the
seeded generators in ``seeded_inputs``, which hold none of the method's
arithmetic.

The oracle is deliberately plain and slow:

* tensors are dense numpy arrays in float64; an abelian symmetry is carried as
  an integer charge label per basis index (``labels.py``), and blocks are only
  formed where the method itself needs them (the SVD truncation, Sec. IV A);
* every contraction is the literal definition from the paper written as one
  ``numpy.einsum`` (``contract.py``);
* the local update follows the eight steps of Sec. V in the paper's order
  (``dmrg3s.py``);
* the Hamiltonians and their exact energies come from an independent route
  (Kronecker products and free-fermion closed forms, ``models.py`` /
  ``exact.py``) so that the DMRG machinery can be pinned against them.

Index conventions (all modules):

* MPS site tensor ``M[s, al, ar]`` of shape ``(d, m_{i-1}, m_i)`` (Sec. II);
* MPO site tensor ``W[s_out, s_in, bl, br]`` of shape ``(d, d, w_{i-1}, w_i)``;
  ``s_out`` is the bra (row) index of the local operator;
* environments ``L[b, a_bra, a_ket]`` and ``R[b, a_bra, a_ket]``, both of shape
  ``(w, m, m)``, with ``L_0 = R_{l+1} = 1`` (Sec. II).
"""
