"""GB300 (sm_103a) steady linearized-Boltzmann solver: fast-spectral hard-sphere collision
operator, upwind transport sweeps, CIS and the synthetic iterative scheme of
arXiv:1612.04488, behind the C ABI of include/lbe.h (liblbe.so)."""
from . import lbe  # noqa: F401
