"""GB300-native aTTN hot path: H_eff application, renormalisation, Lanczos, QR,
disentangler update and sweep in hand-written sm_103a kernels behind the C ABI
of ``include/attn.h``. ``attn`` is the ctypes binding (marshalling only)."""
from . import attn  # noqa: F401
from ._build import build, LIB  # noqa: F401
