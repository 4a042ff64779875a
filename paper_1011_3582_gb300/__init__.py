"""GB300-native FFT-LB for thermal liquid-vapour systems (arXiv:1011.3582).

The compute path is the C-ABI library ``libfftlb.so`` built from ``csrc/``;
``paper_1011_3582_gb300.fftlb`` is its ctypes binding.  Importing this
package does not load the library: ``from paper_1011_3582_gb300 import fftlb``
does, and fails loudly when it has not been built.
"""
__all__ = ["fftlb", "workloads"]
