"""Algorithmic operation and byte counts of the WENO-C operator, per interior
cell and per direction sweep, used for the roofline fractions.

Counting rules: add, subtract, multiply = 1 flop; fused multiply-add = 2;
divide = 1; square root = 1; compares, min/max and selects = 0.  The counts
follow the arithmetic the method needs on its common path (every limiter
factor equal to one, unit fraction sums, no degenerate weights); branches that
only run near bounds are not counted, so the count is a lower bound of the
work done.  Each term names the step it counts.
"""
from __future__ import annotations


def flops_per_cell_dir(N: int, D: int, hllc: bool = False, rk_stage: bool = True) -> int:
    NV = 2 * N + D + 1
    # cons -> prim of the cell (mixture rules, Eq. 27): rho, 1/rho, |rho u|^2,
    # sum A alpha, sum B alpha, u, P
    prim = (N - 1) + 1 + 2 * D + 4 * N + D + 6
    # one WENO5 variable with its own weights (Eq. 15) on both faces:
    # 4 stencil differences, 3 smoothness indicators (9 + 7 + 9),
    # 2 weight sets (19 each), 2 faces x (3 candidates 7 + combination 7)
    full_var = 4 + 25 + 2 * 19 + 2 * 14
    # a volume fraction with the weights of its mass (Eq. 16)
    frac_var = 4 + 2 * 14
    recon = full_var * (N + D + 1) + frac_var * N
    # limiter chain: Eq. 17-18 and Eq. 20 (interior value and theta checks,
    # 4 flops per field, masses and fractions), Eq. 19 sums, V -> U of both
    # faces, Eq. 21 (U^C, psi at average/faces/interior)
    eq17 = 8 * N
    eq19 = 2 * (N - 1)
    eq20 = 8 * N
    v2u = 2 * (5 * N + 3 * D + 2)
    eq21 = 4 * NV + 12 * N + (3 * N + 2 * D + 3)
    limiter = eq17 + eq19 + eq20 + v2u + eq21
    if not hllc:
        # HLL with u-hat from the physical fluxes of Eq. 1: densities
        # 2(N-1); sound speeds of Eq. 2, 6N + 1 a side (P + Pinf, A gamma
        # alpha, product and sum per phase; sum A alpha; rho sum A alpha,
        # divide, square root); wave speeds 4; k = s_L/(s_R - s_L) 2; u-hat 3;
        # per component F_L + k((F_L - F_R) + s_R (U_R - U_L)) 6 plus the two
        # physical fluxes: 2 for masses, fractions and tangential momentum,
        # 4 for the normal momentum and the energy
        flux = 2 * (N - 1) + 2 * (6 * N + 1) + 4 + 2 + 3 + 2 * N * 8 + 10 + (D - 1) * 8 + 10
    else:
        flux = 2 * (N - 1) + 2 * D + 1 + 12 * N + 6 + 4 + 4 * N + 8 * D + 9 \
            + 20 + 3 + 3 * N + 3 * D + 6 + 4 * N + 2 * D + 5 + 12
    # conservative update of Eq. 3 (flux difference, u-hat source term)
    update = 2 * NV + 2 + 2 * N
    # Runge-Kutta combination, spread over the D sweeps of a stage
    rk = (6 * NV) // D if rk_stage else 0
    return prim + recon + limiter + flux + update + rk


def bytes_per_cell_stage(N: int, D: int) -> float:
    """Minimum FP64 state traffic of one SSP-RK3 stage per cell: read U^(k),
    write U^(k+1), and read U^n in stages 2 and 3 (average 8/3 state passes)."""
    NV = 2 * N + D + 1
    return 8.0 * NV * (2 + 3 + 3) / 3.0
