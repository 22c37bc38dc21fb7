"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds input generators only: images, binary masks, formula
DAGs and query streams shaped like the workloads of the paper's evaluation
(Sec. 4: large random / sequential formulas, and the BraTS-like brain-tumour
segmentation on MRI slices).  It contains none of the model checker's
arithmetic; every function here returns plain numpy arrays or plain Python
lists of node records.

A formula is a list of ``Node`` records in topological order (operands refer
to strictly smaller indices) plus a list of root indices.  Operators are named
by strings so that neither side's numeric encoding leaks into the other.
"""
from .formulas import (Node, Formula, OPS, PRIMITIVE_OPS, DERIVED_OPS, NUMBER_OPS,
                       random_dag, sequential_dag, arith_dag, config1_formula,
                       config4_formula, grow_spec_formula, grow_spec_u16_formula,
                       formula_to_records)
from .images import (gaussian_field_image, uniform_image, uniform_image_u16, to_u16,
                     bernoulli_mask, spiral_mask, checkerboard_mask, rings_mask, rings_count,
                     mri_phantom_batch, mri_phantom_batch_parallel, mri_side_lengths,
                     mri_phantom_volume, seed_mask)
from .streams import poisson_queries

__all__ = [
    "Node", "Formula", "OPS", "PRIMITIVE_OPS", "DERIVED_OPS", "NUMBER_OPS", "random_dag",
    "sequential_dag", "arith_dag", "config1_formula", "config4_formula", "grow_spec_formula",
    "grow_spec_u16_formula", "formula_to_records", "gaussian_field_image", "uniform_image",
    "uniform_image_u16", "to_u16", "bernoulli_mask",
    "spiral_mask", "checkerboard_mask", "rings_mask", "rings_count",
    "mri_phantom_batch", "mri_phantom_batch_parallel", "mri_side_lengths", "mri_phantom_volume",
    "seed_mask", "poisson_queries",
]
