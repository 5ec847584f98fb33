"""frx: forward-error-oriented eigenvector refinement with Ozaki-scheme products (GB300).

The compute path lives in the CUDA library ``lib/libfrx.so`` (C ABI in
``include/frx.h``); ``api`` is a thin ctypes binding over it that marshals torch
CUDA tensors.  ``synth`` builds seeded synthetic inputs.  Import ``api`` lazily so
that the input generators work without the built library.
"""
