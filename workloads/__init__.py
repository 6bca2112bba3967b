"""Seeded synthetic inputs for the Sparrow environment step.

This package only produces *input data*: occupancy grids and workload
descriptions (env counts, randomisation ranges, map assignment). It holds none
of the simulator's arithmetic, so both the CPU oracle and the CUDA path can
consume the same inputs without sharing any code of the method itself.
"""

from .maps import make_map, map_start_goal
from .configs import WORKLOADS, workload

__all__ = ["make_map", "map_start_goal", "WORKLOADS", "workload"]
