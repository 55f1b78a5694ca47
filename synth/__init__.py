"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This package holds no arithmetic of the method (no contact geometry, no QP data,
no PDIP or tensor-train step): it only draws the granular scenes and the random
vectors that both sides consume, so that neither side imports the other.
"""
from .scenes import Scene, lattice_scene, column_scene, box_scene, scene_for, SCENES, splitmix64_uniform, normal_vector, random_vector

__all__ = ["Scene", "lattice_scene", "column_scene", "box_scene", "scene_for", "SCENES", "splitmix64_uniform", "normal_vector", "random_vector"]
