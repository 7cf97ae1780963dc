"""GB300 (sm_103a) cross-matrix Krylov projection solver for the implicit
log-density Fokker-Planck systems of arXiv 2511.17634.

The compute path lives in the CUDA library built from ``csrc/`` and is
reached through the C ABI declared in ``include/kp.h``; ``kp`` is its thin
Python binding.  ``synth`` generates the seeded synthetic inputs.
"""
__all__ = ["kp", "synth"]
