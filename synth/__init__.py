"""Seeded synthetic inputs (water boxes with ions, point-charge systems for
molecular dynamics) for tests and benchmarks.

Holds none of the multilevel summation arithmetic: it only places atoms and
assigns charges.  Both the oracle side and the CUDA side take their inputs
from here.
"""
from .water import (TIP3P, WORKLOADS, Workload, make_water_box, replica_boxes,  # noqa: F401
                    replica_sizes, workload, spatial_subsample)
from .ions import make_ion_system  # noqa: F401
