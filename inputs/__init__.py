"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds workload descriptions (grid sizes, boundary kinds, geometry
parameters, physical constants) and seeded random draws (initial-condition
noise, geometry offsets).  It holds none of the method's arithmetic: no
classification, no weights, no stencils, no Poisson solve.  Both the oracle and
the GPU binding consume the plain numbers produced here.
"""
from .configs import (BC_PERIODIC, BC_NOSLIP, BC_FREESLIP, BC_INFLOW, BC_OUTFLOW,
                      GEOM_NONE, GEOM_PLANES, GEOM_CYLINDER, GEOM_SPHERE,
                      GEOM_SINE_WALL, GEOM_TUBES, GEOM_SAMPLED,
                      B_EXACT, B_EULER, B_TAYLOR2, B_EXPLICIT, FLOW_FORCED, FLOW_CONST_FLUX,
                      Case, channel_c1, cylinder_c2, cylinder_c2_io, cylinder_paper, wavy_c3, airway_c4, small_case,
                      couette_case, pipe_case, serving_mix, tanh_faces)
from .generators import initial_field, noise_field, tube_union

__all__ = [n for n in dir() if not n.startswith("_")]
