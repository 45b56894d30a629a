"""FP64 CPU oracle of the yarn BYSDF -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this package.  The CUDA product path never imports it.
The C++ source (``bysdf_oracle.cpp``) follows the paper step by step; this
module only builds it and marshals numpy arrays through ctypes.

Parity unpinned: the paper prints no per-evaluation value, so the composite
BYSDF value itself has no external pin; every building block is pinned by the
tests under ``tests/test_oracle_*.py`` (closed forms, brute force, invariants).
"""
from .oracle import (  # noqa: F401
    NPARAM,
    NPARAM_EXT,
    STOCH_JITTER_NODES,
    STOCH_ROUGH_ENTRY,
    build,
    count_ops,
    eval_records,
    eval_stochastic_records,
    fiber_map,
    fiber_map_tab,
    fresnel,
    geometry,
    ggx_d,
    ggx_g1,
    grad_ext_records,
    grad_records,
    internal_offsets,
    layout,
    lib,
    lobes,
    margin,
    margins,
    MARGIN_CLASSES,
    migration_info,
    migration_texels,
    btdf,
    pdf_records,
    philox4x64,
    ply_occlusion,
    sample_records,
    sample_stochastic_records,
    stoch_nodes,
    trace_yarns,
    vndf_pdf,
    vndf_sample,
)
