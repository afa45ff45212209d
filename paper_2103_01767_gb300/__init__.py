"""GB300-native matrix-free Levenberg-Marquardt ptychography (arXiv 2103.01767).

``synth`` draws seeded synthetic inputs; ``ptylm`` is the thin ctypes binding over the
CUDA library's C-ABI (``include/ptylm.h``).  The binding is imported on demand so that the
input generators stay usable on machines without the built library.
"""
__all__ = ["synth"]
from . import synth  # noqa: E402
