"""GB300 (sm_103a) sliding-window root-MUSIC phase-derivative demodulation (arXiv:1910.11872).

The computation lives in the CUDA library built from ``csrc/`` (C ABI in ``include/rmusic.h``);
``rmusic`` is its ctypes binding and ``synth`` draws seeded synthetic fringe stacks."""

__all__ = ["rmusic", "synth", "build"]
