"""GB300-native subpixel-level 3D Gaussian Splatting for lenticular light-field
displays (CoherentRaster, arXiv 2605.04509).

The renderer lives in a CUDA shared library behind a C ABI
(``include/lfd.h``); ``paper_2605_04509_gb300.lfd`` is its thin ctypes
binding and ``paper_2605_04509_gb300.synth`` draws seeded synthetic inputs.
Importing this package loads neither.
"""
