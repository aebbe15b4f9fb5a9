"""GB300-native streaming inference for detector time series (arXiv 2108.12430).

The compute path lives in the C-ABI shared library built from ``csrc/``
(``libgwstream.so``); ``gwstream`` is its thin ctypes binding.  ``synth``
holds the seeded synthetic-input generators.  Importing this package loads
nothing; the library is opened on first use of ``gwstream.lib()``.
"""
