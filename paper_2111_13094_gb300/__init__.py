"""GB300-native (sm_103a) spatio-directional Gaussian mixtures for path
guiding: weighted, averaged MAP-EM fitting of 5-D mixtures per region, and
conditioned sampling / pdf queries, after Dodik et al., "Path Guiding Using
Spatio-Directional Mixture Models".

The computation lives in the CUDA library libsdmm.so (C ABI:
include/sdmm.h); this package marshals torch tensors into it.  Importing the
package does not load the library; the first call does, and raises if it
cannot be built or loaded.
"""
from ._lib import SdmmError, load  # noqa: F401

__version__ = "0.1.0"


def __getattr__(name):
    # the torch-facing API is imported lazily so that the data generator
    # (paper_2111_13094_gb300.synthetic) can be used without torch/CUDA
    import importlib
    if name.startswith("__"):
        raise AttributeError(name)
    api = importlib.import_module(__name__ + ".api")
    if name == "api":
        return api
    if hasattr(api, name):
        return getattr(api, name)
    raise AttributeError(name)
