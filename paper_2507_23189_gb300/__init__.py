"""GB300 Monte Carlo / Lorenz-Mie photon-transport engine (arXiv 2507.23189).

The per-photon random walk through a turbid suspension (free path, Mie or
Henyey-Greenstein scattering, implicit capture with roulette, index-matched
cuvette walls, side-camera next-event estimate) runs in hand-written sm_103a
CUDA behind the C ABI in include/mcmie.h; this package is its binding.
"""
from . import _native
from .engine import (Batch, Camera, Engine, Geometry, Grid, Medium, MixtureTable, PaperTable, PhaseTable,
                     WeightedTable, auto_frac_bits, camera_image, decode_trace, host_workspace_bytes, image_metrics, philox, run_host,
                     run_params, wait_selftest)
from .checkpoint import append_jsonl, run_record, run_resumable

__all__ = ["Batch", "Camera", "Engine", "Geometry", "Grid", "Medium", "MixtureTable", "PaperTable", "PhaseTable",
           "WeightedTable", "auto_frac_bits", "camera_image",
           "decode_trace", "host_workspace_bytes", "image_metrics", "philox", "run_host", "run_params",
           "wait_selftest", "run_resumable", "run_record", "append_jsonl", "lib"]


def lib():
    """The loaded engine library (build it with paper_2507_23189_gb300.build.build())."""
    return _native.lib()
