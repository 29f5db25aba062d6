"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

It holds no point-in-polygon arithmetic: only random polygon partitions,
hierarchies and point streams. Both the oracle side and the CUDA side take
their inputs from here.
"""
from .partition import UNITS_PER_DEG, PolygonSet, merge_sets, voronoi_partition  # noqa: F401
from .points import Mixture, degenerate_lattice, lattice_to_degrees, uniform_lattice  # noqa: F401
from . import configs  # noqa: F401
