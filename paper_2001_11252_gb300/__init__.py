"""GB300-native resonant-line Monte Carlo radiative transfer (RASCAS hot path).

Thin Python binding over the C ABI declared in ``include/rascas_gb300.h``:
argument marshalling only.  Every step of the transfer runs in the CUDA
library ``_build/librascas_gb300.so`` (built by ``build.py``); importing this
package raises if that library cannot be loaded -- there is no CPU fallback.

PyTorch is used for device memory and streams: tensors passed to the calls
below are handed to the library as raw device pointers on the current torch
stream; numpy arrays are passed as host buffers.
"""
from ._native import (  # noqa: F401
    Context, Stats, Event, RascasError, lib, library_path,
    TALLY_SPECTRUM, TALLY_PEEL_SPECTRA, TALLY_PEEL_IMAGES, TALLY_PEEL_CUBES,
    PK_ACTIVE, PK_ESCAPED, PK_ABSORBED, PK_CAPPED, PK_ERROR,
    DOMAIN_SPHERE, DOMAIN_SLAB, DOMAIN_CUBE, DOMAIN_SHELL, BATCH_PERSISTENT, BATCH_PER_MODEL,
    VOIGT_TASITSIOMI, VOIGT_FADDEEVA,
)
