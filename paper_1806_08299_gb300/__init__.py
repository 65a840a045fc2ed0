"""GB300 (sm_103a) time-tiled acoustic wave library.

The compute path is libwavetile (C ABI in include/wave.h, CUDA sources in
csrc/); `wave` is its ctypes binding, `autograd` wraps it as a
torch.autograd.Function, `inputs` builds seeded synthetic workloads and
`build` compiles the library in-tree.
"""
from . import build, inputs  # noqa: F401
from .wave import Grid, Tuning, WaveError  # noqa: F401
