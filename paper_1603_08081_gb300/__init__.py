"""GB300 (sm_103a) shiftable Fourier-kernel bilateral filter (arXiv 1603.08081).

The C ABI is ``include/fbf.h``; ``paper_1603_08081_gb300.fbf`` is its Python
binding (it loads the CUDA library on import and fails loudly when it is
missing).  ``paper_1603_08081_gb300.synth`` generates the seeded test images.
Importing this package itself loads nothing.
"""
__all__ = ["fbf", "synth", "build"]


def __getattr__(name):
    if name in ("fbf", "synth", "build"):
        import importlib

        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
