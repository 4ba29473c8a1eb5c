"""GB300-native hierarchy-cut-code ray reordering (arXiv 2305.16652).

The compute path is the CUDA library ``csrc/_build/libhcc.so`` (C ABI in
``include/hcc.h``); ``hcc`` is its Python binding and ``gen`` produces the
seeded synthetic inputs.  ``build()`` compiles the library for sm_103a.
"""
from .build import build  # noqa: F401
