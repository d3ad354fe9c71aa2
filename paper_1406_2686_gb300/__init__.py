"""GB300-native hybrid lattice-Boltzmann / finite-difference solver for
viscoelastic two-component flows (Gupta, Sbragaglia & Scagliarini).

The compute path lives in the CUDA library ``libvefd.so`` (sources in
``csrc/``, C-ABI declared in ``include/vefd.h``); ``vefd`` is its thin
ctypes binding and ``inputs`` the seeded synthetic-input generators.
Importing this package loads nothing; ``vefd`` loads the library on first use
and raises if it is missing.
"""

__all__ = ["vefd", "inputs"]
