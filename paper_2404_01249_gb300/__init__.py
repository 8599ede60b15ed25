"""GB300-native inner loop of FireANTs' multi-scale Riemannian-Adam
diffeomorphic registration (arXiv 2404.01249).

The compute lives in ``libfa`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/fa.h``); ``paper_2404_01249_gb300.fa`` is the thin
ctypes binding with the same entry-point names.  ``autograd`` wraps the
warp + LNCC loss and its adjoints as a ``torch.autograd.Function``,
``template`` computes a template gradient over many subjects (all-reduced
across ranks), and ``synth`` draws the seeded synthetic inputs.  The binding is imported lazily so that the generators can
be used on machines without the library; every binding call raises if the
CUDA library is missing.
"""
import importlib

__all__ = ["fa", "synth", "autograd", "template"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
