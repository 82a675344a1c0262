"""Batched X-Drop seed extension (arXiv 2304.08662) on GB300: CUDA kernels for sm_103a
behind the C ABI of include/xdrop.h, with a thin ctypes binding (``xdrop``)."""
from . import xdrop  # noqa: F401
