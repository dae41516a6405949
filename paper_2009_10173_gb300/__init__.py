"""GB300 (sm_103a) model-based AR-OAM inversion: slab builder, A / A^T and the
LSQR / FISTA solvers behind the C-ABI library ``liboam.so``."""
