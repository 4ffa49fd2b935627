"""GB300-native batched fitness evaluation for stack-based genetic programming.

Implements the evaluation hot path of arXiv 2110.11226 ("Accelerating Genetic
Programming using GPUs"): a whole population of prefix-list programs is
evaluated over every row of a column-major FP32 dataset with the weighted loss
fused into the evaluation, then tournament selection runs on the device.

Importing the package loads nothing native; ``paper_2110_11226_gb300.gp``
loads the CUDA library (``libgp.so``) and raises if it is missing.
"""
__all__ = ["synth", "gp"]
