"""GB300-native Online FISTA for sparse SAR (arXiv 2603.08582).

The compute path lives in libosar.so (CUDA, sm_103a); `osar` is its ctypes
binding, `synth` the seeded input generator, `build` the in-tree build step.
"""

__all__ = ["osar", "synth", "build"]
