"""B300-native box-tracking hot path (OmniTrack tracking phases, Section V-A).

The CUDA library libomt.so does all the work; ``omt`` is its ctypes binding
and ``synth`` the seeded synthetic-input generator.
"""
from . import omt  # noqa: F401

__all__ = ["omt"]
