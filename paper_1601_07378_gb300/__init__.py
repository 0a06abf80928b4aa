"""GB300-native V_loc|psi> library: the local-potential action of plane-wave
Kohn-Sham codes via a compact 3-D FFT with plane-wave load balancing
(Gao, Mo, Fang & Wang, arXiv:1601.07378), as hand-written sm_103a CUDA
behind a C ABI (include/vloc.h).

The CUDA library is loaded on first use (``vloc.load()``); importing the
package does not require a GPU.
"""
__version__ = "0.1.0"
