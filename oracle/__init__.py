"""FP64 CPU oracle of the IBP objective bound (test infrastructure only).

Imported only by the tests, the smoke check and the CPU-baseline leg of the
benchmark.  Shares no code with the CUDA library.
"""
from .reference import *  # noqa: F401,F403
from .reference import (  # noqa: F401
    Sensitivities, Bound, IslandingContingency, sensitivities, ptdf, lodf, bound,
    bus_box, cost_interval, imbalance_interval, imbalance_matrix, base_terms, ctg_terms,
    ctg_flows, all_ctg_flows, objective_point, grad_hi, grad_hi_ratings, grad_lo, linear_bound, paper_mode_flows,
    paper_ctg_matrices, outage_ptdf, relu_chain_interval, viol_interval, incidence,
    reduced_admittance,
)
