"""GB300-native (sm_103a) hot path of the RBM-Chebyshev method for spin
spectral functions (Hendry, Chen, Weinberg, Feiguin, arXiv:2103.08804).

The compute lives in the C-ABI library ``libchebrbm.so`` (hand-written CUDA,
declared in ``include/chebrbm.h``); ``paper_2103_08804_gb300.api`` is the thin
Python binding over it.  Importing this package does not load the library:
``synth`` (seeded synthetic inputs) works without a GPU.
"""

__all__ = ["api", "synth", "build", "driver", "autograd"]


def __getattr__(name):
    if name in ("api", "synth", "build", "driver", "autograd"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
