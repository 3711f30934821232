"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *builds problem data* (matrices, vectors, cone lists) from
seeded random numbers.  It holds none of the solver's arithmetic: no
projection, no linear solve, no iteration.  Both the CPU oracle and the CUDA
path consume what it produces.

Problem form (paper Sec. 2.1, Eq. conic-standard):

    minimize  1/2 x'Px + q'x   s.t.  Ax + s = b,  s in K

with K a Cartesian product of cones listed in row order.
"""
from .problem import (ConicProblem, ZERO, NONNEG, BOX, SOC, PSD, CONE_NAMES,
                      svec_index, svec_len)
from .generators import (erdos_renyi, maxcut_problem, lovasz_problem,
                         socp_problem, covsteer_problem, linsys_instance,
                         clustered_symmetric, random_graph_batch,
                         cycle_graph, complete_graph, empty_graph)
from .classes import (lyapunov_problem, robust_kalman_problem, robust_mpc_problem,
                      hurwitz_matrix, kalman_matrices, mpc_tightening)
from .steering import cs_problem, cs_double_integrator_problem, double_integrator

__all__ = [
    "ConicProblem", "ZERO", "NONNEG", "BOX", "SOC", "PSD", "CONE_NAMES",
    "svec_index", "svec_len", "erdos_renyi", "maxcut_problem",
    "lovasz_problem", "socp_problem", "covsteer_problem", "linsys_instance",
    "clustered_symmetric", "random_graph_batch", "cycle_graph",
    "complete_graph", "empty_graph", "lyapunov_problem", "robust_kalman_problem",
    "robust_mpc_problem", "hurwitz_matrix", "kalman_matrices", "mpc_tightening",
    "cs_problem", "cs_double_integrator_problem", "double_integrator",
]
