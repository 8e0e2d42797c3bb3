"""B300-native batched 3D Gaussian Splatting renderer.

The rendering hot path (projection + SH colour + cull, depth sort, tile
binning, front-to-back compositing) runs in hand-written sm_103a CUDA kernels
inside ``libgs_b300.so`` behind the C ABI declared in ``include/gs.h``.
``paper_2510_15352_b300.gs`` is the Python binding (argument marshalling
only); importing it loads the library and fails loudly if it is missing.
``paper_2510_15352_b300.synth`` holds the seeded input generators.
"""
__all__ = ["gs", "synth"]
