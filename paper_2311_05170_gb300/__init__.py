"""GB300 (sm_103a) library for the local parallel two-grid finite element method for the
transient triple-porosity Navier-Stokes model (Algorithm 3): a C ABI (include/tpns.h)
implemented by hand-written CUDA kernels, and a thin ctypes binding."""
from .native import Solver, TpnsError, batch_step, load  # noqa: F401
