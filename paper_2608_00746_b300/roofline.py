"""Algorithmic operation and byte counts of the WENO-C operator, per interior
cell and per direction sweep, and the peaks they are held against.

The flop counts are the oracle's: its counting build (every FP64 operation of
the definition counted by step, on the common path of a smooth state) writes
``op_counts.json`` beside this module (``python -m oracle.op_count``; a CPU
test re-derives the file).  Add, subtract, multiply, divide and square root
are 1 flop each, comparisons 0; each step is taken as often per cell and
direction as the method needs it (one cons -> prim, the smoothness
indicators of the independently weighted variables once, candidates of every
variable on both faces, the weights, limiter chain, flux and update as
defined).  The kernels compute the same results with fewer operations in
places (one division per weight set, indicators shared by both faces), so
the counts are the work of the method as the paper states it, not the
instructions a kernel issues.
"""
from __future__ import annotations

import json
import os

_COUNTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "op_counts.json")
_cache = None

# Unit-count peaks at the maximum SM clock (2032 MHz) on 148 SMs: FP64 2 DFMA
# per clock per SM, FP32 128 FFMA per clock per SM, 2 flops each.
SM_MHZ = 2032.0
PEAK_FP64_TFLOPS = 2 * 2 * 148 * SM_MHZ * 1e6 / 1e12
PEAK_FP32_TFLOPS = 128 * 2 * 148 * SM_MHZ * 1e6 / 1e12
# the surrogate (reading 18): 30 -> 64 -> 64 -> 64 -> 9 multiply-adds per face side
MLP_FLOPS_PER_FACE_SIDE = 2 * (30 * 64 + 64 * 64 * 2 + 64 * 9)


def _counts():
    global _cache
    if _cache is None:
        with open(_COUNTS) as fh:
            _cache = {(c["N"], c["D"], c["flux"]): c for c in json.load(fh)["counts"]}
    return _cache


def entry(N: int, D: int, flux: str = "hll") -> dict:
    key = (N, D, flux)
    if key not in _counts():
        raise KeyError(f"no oracle op count for N={N}, D={D}, flux={flux}")
    return _counts()[key]


def flops_per_cell_dir(N: int, D: int, flux: str = "hll") -> float:
    """FP64 flops of one cell in one direction sweep, the Runge-Kutta
    combination's share included."""
    return entry(N, D, flux)["flops_per_cell_dir"]


def mixed_split(N: int, D: int, flux: str = "hll"):
    """(FP64, FP32) flops per cell and direction of the mixed-precision form:
    FP64 for pressure recovery, the limiter chain with its face states, the
    update and the Runge-Kutta combination; FP32 for the indicators, weights,
    candidates, combination and flux."""
    e = entry(N, D, flux)
    return e["mixed_fp64_flops_per_cell_dir"], e["mixed_fp32_flops_per_cell_dir"]


def bytes_per_cell_stage(N: int, D: int) -> float:
    """Minimum FP64 state traffic of one SSP-RK3 stage per cell: read U^(k),
    write U^(k+1), and read U^n in stages 2 and 3 (average 8/3 state passes)."""
    NV = 2 * N + D + 1
    return 8.0 * NV * (2 + 3 + 3) / 3.0
