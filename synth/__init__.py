"""Seeded synthetic inputs for the pSRM EM iteration.

This package only draws random numbers and assembles data of the shapes the
paper works with; it holds none of the EM method's arithmetic.  Both the FP64
oracle (``oracle/``) and the CUDA path (through ``bench.py`` and the tests)
take their inputs from here.
"""
from .planted import (  # noqa: F401
    CONFIGS,
    PlantedSpec,
    config_spec,
    draw_voxel_counts,
    planted_subject,
    planted_dataset,
    random_orthonormal,
    initial_mappings,
)
