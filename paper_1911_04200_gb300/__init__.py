"""jsim: exact all-pairs Jaccard similarity on one GB300 GPU.

The method is SimilarityAtScale (arXiv 1911.04200, Sec. III): batched
indicator-matrix rows, zero-row filtering, 64-bit bitmask words and an
AND+popcount semiring product, here as hand-written sm_103a CUDA kernels
behind the C-ABI in ``include/jsim.h``.

Submodules are imported lazily so that ``paper_1911_04200_gb300.synth`` (the
seeded input generator) can be used without loading the CUDA library.
"""

__all__ = ["jsim", "synth", "build_native"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
