"""GB300 (sm_103a) implementation of distributed Affine Body Dynamics with
consensus ADMM.  The compute path lives in libabd.so (C ABI: include/abd.h);
`abd` is its Python binding, `scenes` the seeded synthetic inputs."""
from . import scenes  # noqa: F401

__all__ = ["scenes", "abd", "build"]
