"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the CUDA path's tests/bench and the oracle; it holds
none of the method's arithmetic (no convolution, no decomposition): it only
draws scenes and noise.
"""
from .scenes import (  # noqa: F401
    SEED, config_rng, line_1d_bumps, line_1d_scatterers, image_2d_scene,
    batch_lines, deconv_scene_2d, add_noise_snr, real_noise, paper_example_1d, paper_example_2d,
    rsvd_omega_blocks,
)
