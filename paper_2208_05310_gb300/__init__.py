"""GB300-native DGSEM time step of the relaxed non-isothermal Navier-Stokes-Korteweg
equations (Keim, Munz & Rohde, arXiv 2208.05310).

The compute path is libdgk.so (hand-written CUDA for sm_103a behind the C ABI of
include/dgk.h); `dgk` is its Python binding and `inputs` the seeded synthetic inputs.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "dgk"]
