"""GB300 (sm_103a) implementation of the hot path of arXiv 2401.16322: the 2D acoustic PML
wave operator H (Eq. 1) and the Faber, Krylov, HORK, RK3-2, RK4-4 and leap-frog time
integrators, as fused CUDA kernels behind the C ABI of include/ewave.h."""
from .ewave import Batch, EwaveError, Model, load_library  # noqa: F401
