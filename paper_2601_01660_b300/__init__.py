"""Deep Gaussian Shadow Maps on one B300 (sm_103a).

The hot path of "Animated 3DGS Avatars in Diverse Scenes with Consistent
Lighting and Shadows" (Secs. 3.2-3.5): the closed-form DGSM build over an
octahedral atlas of radial shells, receiver attenuation, and the SH probe
fit + per-Gaussian radiance transfer.  All compute runs in libdgsm.so
(hand-written CUDA behind the C ABI of include/dgsm.h); this package only
binds it.  `scenes` holds the seeded synthetic input generators.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "native"]


def native():
    """Import the CUDA binding (raises ImportError if libdgsm.so is not built)."""
    from . import _native
    return _native
