"""SV-MPR gap filling on GB300 (Lach & Zukovic, arXiv 2212.01317).

The method runs in libmpr.so (hand-written sm_103a CUDA behind the C-ABI in
include/mpr.h); ``mpr`` is its ctypes binding and ``synth`` the seeded input
generators. There is no CPU fallback.
"""
from . import mpr, synth  # noqa: F401
from .mpr import GapFiller, MprError  # noqa: F401

__all__ = ["mpr", "synth", "GapFiller", "MprError"]
