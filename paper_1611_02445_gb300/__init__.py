"""GB300-native sparse-tile D3Q19 lattice-Boltzmann step (Tomczak & Szafran).

The compute path is the C-ABI library ``liblbm_gb300.so`` (hand-written CUDA for
sm_103a); ``paper_1611_02445_gb300.lbm`` is its thin ctypes binding. Importing the
package does not load the library; the binding loads it on first use and raises if
it is missing.
"""
__all__ = ["inputs", "lbm"]
