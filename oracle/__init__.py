"""FP64 CPU oracle for the batched GN/LM solve and its implicit-differentiation backward.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of what
the paper's layer computes (Eq. 1 objective, the GN/LM iteration of Sec. 2, the implicit
derivative of Eq. 3 / Prop. 1).  Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it.  It shares no code with the CUDA path: derivatives here come from
autograd through the residual definitions, linear systems are solved by LAPACK (torch.linalg) or
SciPy's sparse LU, and nothing is blocked, fused or reordered beyond the definitions.
"""
