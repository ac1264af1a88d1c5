"""GB300-native efficient permutation two-sample tests (energy distance / Gaussian MMD).

The compute path is the C-ABI library ``libept.so`` (hand-written sm_103a CUDA,
declared in ``include/ept.h``); ``ept`` is its thin ctypes binding.  Importing this
package does not load the library: ``from paper_2406_06488_gb300 import ept``
does, and fails loudly if it has not been built.
"""
__all__ = ["ept", "workloads"]
