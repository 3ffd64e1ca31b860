"""FP64 CPU oracle for the RIOT inner loop (test infrastructure only).

A plain, slow, obviously correct restatement of the method of Bousserez,
Guerrette & Henze (arXiv:1906.01413): the Lorenz-96 model, its tangent-linear
and adjoint integrations in plain C (``l96.c``), and the 4D-Var / RIOT linear
algebra in numpy FP64 (``riot.py``).  It shares no code with the CUDA
library.  Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import it; the library itself never does.
"""
