"""B300-native unrolled COSMO (deep-unfolded ADMM conic solver) hot path.

The compute path is ``libcosmo_du.so`` (hand-written sm_103a CUDA kernels
behind the C ABI of ``include/cosmo_du.h``); this package is its Python
binding.  Importing the package does not load the library; the first call
that needs it does, and fails loudly if it has not been built.
"""
from ._abi import CosmoError, lib, LIB_PATH  # noqa: F401


def __getattr__(name):
    # lazy: keep `import paper_2606_13825_b300` free of torch / CUDA work
    if name in ("CosmoBatch", "CosmoUnroll", "RhoFromLog", "AlphaBroadcast",
                "unrolled_residual_loss", "psd_project", "psd_dk_backward", "pack",
                "validate", "default_options", "WarmStart", "WarmStartNet", "ws_sizes",
                "PolicyUnroll", "HyperPolicy", "policy_sizes", "policy_default_l0"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
