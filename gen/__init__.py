"""Seeded synthetic SC-DCOPF cases shared by the oracle tests, the GPU tests and the bench.

This package only *draws* inputs (networks, devices, costs, boxes, contingency
lists).  It holds none of the interval-bound arithmetic: the oracle and the CUDA
library each compute every sensitivity and bound on their own.
"""
from .cases import (  # noqa: F401
    Case,
    CONFIG_SIZES,
    make_case,
    make_config,
    make_network_case,
    make_ragged_batch,
    find_bridges,
    split_boxes,
)
