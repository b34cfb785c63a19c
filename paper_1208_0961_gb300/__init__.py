"""GB300-native test-particle transport (arXiv:1208.0961, CuBA): the per-time-step
stream / reflect / bin / 2->2 collide update as hand-written sm_103a CUDA behind
the C ABI of include/cuba.h, with a thin Python binding (``cuba``)."""
from . import cuba  # noqa: F401
