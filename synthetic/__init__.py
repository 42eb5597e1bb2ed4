"""Seeded synthetic inputs (meshes, friction fields, random vectors) shared by the
oracle tests and the CUDA path.  Holds no part of the method's arithmetic."""
from . import rng, meshes, friction  # noqa: F401
