"""Seeded synthetic workloads shared by the CUDA path, the oracle, the tests and the bench.

Nothing in this package computes a step of the pose-cost method (no rasterisation, no
per-pixel cost table, no residuals, derivatives or solver steps). It only builds inputs:
labelled triangle meshes, camera models, poses and observed range images. The observed
range images come from an analytic ray cast of the synthetic *world* (solid boxes, a
heightfield), which plays the part of the physical sensor; the method itself only ever
sees the tessellated *map* mesh.
"""
from .scenes import *  # noqa: F401,F403
