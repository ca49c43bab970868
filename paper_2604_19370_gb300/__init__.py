"""GB300-native quasi-implicit ADS wildfire time step (arxiv 2604.19370).

The compute path is libwf.so (CUDA, sm_103a) behind the C ABI of
include/wf.h; `wf` is its thin ctypes binding and `build` compiles it.
"""
from . import build  # noqa: F401
