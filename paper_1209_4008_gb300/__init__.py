"""GB300-native SU(3) lattice gauge fixing (checkerboard overrelaxation).

The compute path is the C-ABI CUDA library ``libgf.so`` (sources in ``csrc/``,
declared in ``include/gf.h``); ``gf`` is its thin ctypes binding.  ``synth``
builds seeded synthetic input fields.
"""
