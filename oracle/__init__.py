"""CPU oracle (fp64, plain C) for the fluorescent participating-media light tracer.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs are the only callers. The product path (paper_1706_03024_gb300) never imports it.
"""
from .oracle import (  # noqa: F401
    COUNTER_NAMES, adjoint, build, lib, optical_depth, majorant, philox, render, render_camera,
    sample_emission, sigma_t_at, iso_dir, cosine_dir,
)
