"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds random-number generation only and none of the method's
arithmetic: raw normal deviates for the initial tree tensors, random Lanczos
start vectors and random link operators for stand-alone effective-Hamiltonian
tests. Both sides receive the same arrays; each side then does its own
isometrisation, renormalisation and contraction.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter mode: deviate ``i`` of stream
``(seed, stream)`` is ``mix64(key + (i + 1) * GOLDEN)`` with
``key = mix64(seed * GOLDEN ^ mix64(stream + 1))``. Uniforms take the top 53
bits; normals come from the Box-Muller transform on consecutive pairs.
"""
from .synth import (  # noqa: F401
    GOLDEN,
    mix64,
    uniform,
    normal,
    raw_tree_tensors,
    random_vector,
    random_operators,
)
