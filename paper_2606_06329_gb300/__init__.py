"""GB300-native (sm_103a) hot path of the MeCuCo local mean-curvature estimator
(arXiv 2606.06329): kNN, patch centring, truncated SVD through the k x k Gram,
and the Fast-mode estimator, as CUDA kernels behind the C ABI in
include/mecuco.h.  ``api`` is the thin Python binding (``autograd`` wraps the
curvature and its adjoint as a torch.autograd.Function); ``synth`` holds the
seeded synthetic workloads; ``build`` compiles the library in tree; ``shard``
splits the query rows over ranks and gathers kappa; ``report`` prints the
curvature-fidelity tables.

Importing the package loads nothing; ``api`` loads lib/libmecuco.so on first
use and raises if it has not been built.
"""
__all__ = ["api", "synth", "build", "autograd", "shard", "report"]


def __getattr__(name):
    if name in ("api", "synth", "build", "autograd", "shard", "report", "_native"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
