"""GB300-native in-place samplesort (IPS4o) and radix sort (IPS2Ra).

The compute path lives in the CUDA library built from ``csrc/`` (C-ABI
declared in ``include/ipsgpu.h``); ``ipsgpu`` is its thin ctypes binding and
``inputs`` makes seeded synthetic inputs.  Importing this package loads
nothing; the binding loads the library on first use and raises if it is
missing.
"""
