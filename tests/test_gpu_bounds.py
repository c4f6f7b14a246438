"""Bounds and unity sum as Eq. 8 and Eq. 19 state them, in every precision
mode, at the faces the sweep hands to the Riemann solver (wc_faces: the
limited conservative states U^L_{i+1/2}, U^R_{i-1/2} of each direction) and
at the cell averages after every step.

Faces: masses >= 0 and fractions in [0, 1] with no slack (R13 sets the
rounding residue of the blends below 0 to 0; blends of values <= 1 cannot
round above 1), and |sum_p alpha_p - 1| <= 2N 2^-53 (Eq. 19 divides each
fraction by the face sum, one rounding each; Eq. 20-21 scale all phases
alike; the check's own summation adds N - 1 roundings at most).

Cell averages: the unity sum to the rounding of the steps taken (the
method normalises the faces, not the averages, so each step's stage sums
round and nothing removes it): 2N 2^-53 per step on top of the initial
state's own.  Masses >= 0 and fractions in [0, 1] with no slack at the
time step for which Sec. 4.2 guarantees them, CFL <= 1/12 (the
Gauss-Lobatto weight), with R13 removing the rounding residue.  At the
workloads' own CFL numbers (0.2, 0.5) the scheme may leave the bounds by
itself (reading R13: that excursion stays and the next limiter takes the
cell to first order), so there the faces and the sums are checked.

The learned mode runs an untrained surrogate with nearly every learned
weight accepted (tau = 1: within the stencil's range of the plain
reconstruction), so the bounds rest on the limiter chain alone."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_00746_b300 import inputs, surrogate

from gpu_util import grids, to_dev

pytestmark = pytest.mark.gpu
U53 = 2.0 ** -53

CASES = {
    "slab_1d_hllc": (lambda: inputs.interface_advection_1d(n=200), 30),
    "shock_bubble_2d": (lambda: inputs.shock_bubble_2d(nx=128, ny=64, seed=5), 20),
    "circles_2d_n3": (lambda: inputs.circles_shock_2d(shape=(96, 80), seed=5, ncirc=6,
                                                      rmin_cells=4, rmax_cells=14), 20),
    "spheres_3d": (lambda: inputs.spheres_shock_3d(shape=(30, 24, 20), seed=1, nsph=4,
                                                   rmin_cells=3, rmax_cells=7), 8),
}


def _sum(alpha):
    s = alpha[0].copy()
    for p in range(1, alpha.shape[0]):
        s = s + alpha[p]
    return s


def _check_faces(F, A, N, d, where):
    """Faces F of the cell state A: where every cell average is inside its
    bounds, every face value is too.  A cell whose average the scheme took
    outside a bound (possible above CFL 1/12) has theta = 0 in Eq. 18 and
    Eq. 20: its faces are its averages (R13 keeps such values)."""
    F = F.cpu().numpy()
    a0 = N + d + 1
    out = (A[:N] < 0.0).any(0) | (A[a0:] < 0.0).any(0)   # theta = 0 here
    ins = ~out & ~(A[a0:] > 1.0).any(0)
    m, a = F[:N][:, ins], F[a0:][:, ins]
    assert m.min() >= 0.0, (where, "mass", m.min())
    assert a.min() >= 0.0 and a.max() <= 1.0, (where, a.min(), a.max() - 1.0)
    err = np.abs(_sum(a) - 1.0).max()
    assert err <= 2 * N * U53, (where, "face sum", err / U53)
    if out.any():
        for v in list(range(N)) + list(range(a0, a0 + N)):
            assert np.array_equal(F[v][out], A[v][out]), (where, "outside cell", v)


@pytest.mark.parametrize("cfl", ["sufficient", "workload"])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "learned"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bounds_and_unity_sum_exact(gpu, name, mode, cfl):
    make, steps = CASES[name]
    case = make()
    N, d = case.N, case.dim
    go, g = grids(case, precision=mode)
    U0 = oracle.prim_to_cons(go, case.V)
    U = to_dev(U0)
    if mode == "learned":
        S = surrogate.Surrogate(seed=5)
        g.set_mlp(S.params, tau=1.0)
    g.bind(U)
    c = 1.0 / 12.0 if cfl == "sufficient" else (case.cfl or 0.2)
    a0 = N + d + 1
    base = np.abs(_sum(U0[a0:]) - 1.0).max()
    worst = 0.0
    for step in range(1, steps + 1):
        A = U.cpu().numpy()
        for ax in range(d):
            UL, UR = g.faces(U, ax)
            _check_faces(UL, A, N, d, (step, ax, "L"))
            _check_faces(UR, A, N, d, (step, ax, "R"))
        g.rk_step(cfl=c)
        A = U.cpu().numpy()
        al = A[a0:]
        if cfl == "sufficient":
            assert A[:N].min() >= 0.0, (step, "cell mass", A[:N].min())
            assert al.min() >= 0.0 and al.max() <= 1.0, (step, al.min(), al.max() - 1.0)
        err = np.abs(_sum(al) - 1.0).max()
        worst = max(worst, (err - base) / step)
        assert err <= base + 2 * N * U53 * step, (step, err / U53)
    g.sync_status()
