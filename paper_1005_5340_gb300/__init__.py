"""GB300 (sm_103a) implementation of the iterative polarizability solve of
Koval, Foerster and Coulaud (arXiv:1005.5340): restarted GMRES on
(1 - chi0(omega) K) X = chi0(omega) d with chi0 and K applied matrix-free by
hand-written CUDA kernels behind a C boundary (include/tddft.h).

``synth`` draws seeded synthetic molecules; ``tddft`` is the binding of the
CUDA library.  Neither is imported here, so that ``synth`` works without a
build of the library.
"""
