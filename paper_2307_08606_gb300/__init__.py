"""GB300-native sharing-ADMM (ASADMM) radar imaging: the per-iteration hot path
of Eq. 3 with Algorithm 1, as hand-written sm_103a CUDA kernels behind the C ABI
in include/sadmm.h.  This package holds the build step and the ctypes binding;
it never falls back to a CPU path."""
from .build import build, LIB

__all__ = ["build", "LIB", "load", "Solver"]


def load():
    from .binding import load as _load
    return _load()


def __getattr__(name):
    if name in ("Solver", "binding"):
        import importlib
        mod = importlib.import_module(__name__ + ".binding")
        return mod if name == "binding" else mod.Solver
    raise AttributeError(name)
