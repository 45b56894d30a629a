"""GB300-native yarn BYSDF ("A Multi-scale Yarn Appearance Model with Fiber
Details"): eval / sample / pdf / backward of the yarn-level BYSDF at ray-yarn
hit records, as CUDA kernels for sm_103a behind the C ABI of include/bysdf.h.

`inputs` (seeded workloads) needs only numpy; `api` needs torch and the built
libbysdf.so and raises if the library is missing (there is no CPU fallback).
"""
from . import build, inputs  # noqa: F401

__all__ = ["build", "inputs", "api"]


def __getattr__(name):
    if name == "api":
        from . import api
        return api
    raise AttributeError(name)
