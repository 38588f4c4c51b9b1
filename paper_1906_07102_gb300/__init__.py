"""Least-misfit gridding and degridding on GB300 (sm_103a).

The compute path lives in the CUDA library ``_lib/liblmg.so`` (sources in ``csrc/``,
C ABI in ``include/lmg.h``); ``lmg`` is the thin ctypes binding that the tests and the
benchmark call. ``synthetic`` draws the seeded synthetic inputs. Importing this package
does not load the CUDA library; ``lmg`` loads it on first use and raises if it is missing.
"""
__all__ = ["lmg", "synthetic"]
