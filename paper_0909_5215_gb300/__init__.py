"""GB300-native batched hyperdynamics for AFM frictional sliding (Kim & Falk).

`model` builds seeded inputs; `hd` is the thin binding over the C-ABI
library (libhdslide.so) whose CUDA kernels run every step of the path.
"""
from . import model  # noqa: F401
