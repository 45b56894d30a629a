"""GB300-native yarn BYSDF ("A Multi-scale Yarn Appearance Model with Fiber
Details"): eval / sample / pdf / backward of the yarn-level BYSDF at ray-yarn
hit records, as CUDA kernels for sm_103a behind the C ABI of include/bysdf.h.

Submodules: `inputs` (seeded workloads, numpy only), `api` (PyTorch binding;
needs the built libbysdf.so and raises if it is missing -- there is no CPU
fallback), `build` (nvcc build), `dist` (record sharding across ranks).
"""
