"""GB300-native implicit filter for spatial spectra (sm_103a CUDA behind a C ABI).

The compiled library libifilt.so (include/ifilt.h) does all the work: mesh
preparation, the batched and plain conjugate-gradient solves, and spectra.
`api` is its Python binding.
"""

from . import api  # noqa: F401
