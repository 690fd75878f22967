"""GB300-native MPLP++ (Handshake dual block-coordinate ascent) solver.

The compute path is the C-ABI library built from ``csrc/`` (CUDA for sm_103a);
``solver`` and ``_lib`` are thin ctypes bindings over it.  Importing this
package loads nothing; the library is loaded on first use and its absence is an
error, never a fallback.
"""
__all__ = ["workloads"]
