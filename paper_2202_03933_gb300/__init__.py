"""GB300 (sm_103a) implementation of segment-based 3D mortar integration.

Mayr & Popp, "Scalable computational kernels for mortar finite element
methods" (arXiv 2202.03933): mortar matrices D and M (Sec. 2.2), segment-based
integration (Algorithm 1), binned contact search (Algorithm 2) and the
gradient of the weighted gap functional, in hand-written CUDA behind the C ABI
of ``include/mortar.h``.  ``mortar`` is the Python binding, ``inputs`` the
seeded synthetic interface generator, ``build`` compiles the library.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("mortar", "inputs"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
