"""GB300-native Yee + UPML FDTD for PCB power integrity.

The compute path is the CUDA library ``libfdtd.so`` (sources in ``csrc/``,
C-ABI declared in ``include/fdtd.h``); this package is its thin ctypes
binding.  ``workloads`` builds the seeded synthetic inputs.
"""
