"""Invariants of the CUDA path in every precision mode: consistency of
reduction (absent phase, bit for bit), unity sum, bounds, equilibrium across an
isolated interface, conservation, and the mixed mode's L1 distance to the FP64
oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_00746_b300 import inputs, wenoc

from gpu_util import grids, l1_group, to_dev

pytestmark = pytest.mark.gpu
MODES = ["fp64", "mixed"]
# Unity sum of the cell averages: 2N 2^-53 per step on top of the initial
# state's own (Eq. 19 normalises faces, not averages, so each step's
# rounding stays; tests/test_gpu_bounds.py states the reading).  Bounds hold
# with no slack (R13).
U53 = 2.0 ** -53


def _sum_err(a):
    s = a[0].copy()
    for p in range(1, a.shape[0]):
        s = s + a[p]
    return np.abs(s - 1.0).max()


@pytest.mark.parametrize("mode", MODES)
def test_absent_phase_bit_identical(gpu, mode):
    """Sec. 3.4: an N-phase run with a phase absent reproduces the (N-1)-phase
    run bit for bit, and the absent phase stays exactly zero."""
    c2 = inputs.interface_advection_1d(n=160)
    c3 = inputs.interface_advection_1d(n=160, absent_phase=True)
    go2, g2 = grids(c2, precision=mode)
    go3, g3 = grids(c3, precision=mode)
    U2 = to_dev(oracle.prim_to_cons(go2, c2.V))
    U3 = to_dev(oracle.prim_to_cons(go3, c3.V))
    g2.bind(U2)
    g3.bind(U3)
    keep, absent = [0, 1, 3, 4, 5, 6], [2, 7]
    assert torch.equal(U3[keep], U2)
    assert torch.equal(g3.rhs(U3)[keep], g2.rhs(U2))
    for _ in range(20):
        d2 = g2.rk_step(cfl=0.5, want_dt=True)
        d3 = g3.rk_step(cfl=0.5, want_dt=True)
        assert d2 == d3
    assert torch.equal(U3[keep], U2)
    assert not U3[absent].any()


def test_absent_phase_bit_identical_2d_table1(gpu):
    c5 = inputs.multiphase_advection_2d(n=48, nphase=5)
    c4 = inputs.multiphase_advection_2d(n=48, nphase=4)
    _, g5 = grids(c5)
    go4, g4 = grids(c4)
    go5, _ = grids(c5)
    U5 = to_dev(oracle.prim_to_cons(go5, c5.V))
    U4 = to_dev(oracle.prim_to_cons(go4, c4.V))
    g5.bind(U5)
    g4.bind(U4)
    g5.rk_step(dt=1e-3, nsteps=10)
    g4.rk_step(dt=1e-3, nsteps=10)
    keep = [0, 1, 2, 3, 5, 6, 7, 8, 9, 10, 11]
    assert torch.equal(U5[keep], U4) and not U5[[4, 12]].any()


@pytest.mark.parametrize("mode", MODES)
def test_equilibrium_bounds_conservation_1d(gpu, mode):
    """Isolated air/water interface (config-1 shape): u and P uniform, fractions
    in [0, 1] summing to one, mass/momentum/energy conserved (periodic)."""
    c = inputs.interface_advection_1d(n=200)
    go, g = grids(c, precision=mode)
    U0 = oracle.prim_to_cons(go, c.V)
    U = to_dev(U0)
    g.bind(U)
    tot0 = U.sum(dim=1)
    g.rk_step(cfl=0.5, nsteps=50)
    g.sync_status()
    V = g.cons_to_prim(U).cpu().numpy()
    scale = 1e5 + max(c.pinf)
    assert np.abs(V[2] - 1.0).max() < 5e-11
    # FP64: the rho E round-off floor; mixed: FP32 flux remainders on top
    assert np.abs(V[3] - 1e5).max() / scale < (1e-14 if mode == "fp64" else 1e-13)
    A = U.cpu().numpy()
    a = A[4:]
    assert A[:2].min() >= 0.0 and a.min() >= 0.0 and a.max() <= 1.0
    assert _sum_err(a) <= _sum_err(U0[4:]) + 2 * 2 * U53 * 50
    tot = U.sum(dim=1)
    rel = ((tot - tot0).abs() / U.abs().sum(dim=1).clamp_min(1e-300)).cpu().numpy()
    assert (rel[:5] < 1e-13).all(), rel


def test_mixed_mode_l1_vs_fp64_oracle(gpu):
    """FP32 reconstruction and flux with FP64 limiter factors, normalisation,
    pressure and update stay within 1e-5 relative L1 of the FP64 oracle."""
    case = inputs.shock_bubble_2d(nx=128, ny=64, seed=5)
    go, g = grids(case, precision="mixed")
    U_or = oracle.prim_to_cons(go, case.V)
    U = to_dev(U_or)
    g.bind(U)
    for _ in range(10):
        U_or, dt = oracle.rk3_step(go, U_or, cfl=0.2)
        g.rk_step(dt=dt)
    A = U.cpu().numpy()
    err = l1_group(A, U_or, case.N, case.dim)
    assert (err <= 1e-5).all(), err
    a = A[-2:]
    assert A[:2].min() >= 0.0 and a.min() >= 0.0 and a.max() <= 1.0
    assert _sum_err(a) <= _sum_err(oracle.prim_to_cons(go, case.V)[-2:]) + 2 * 2 * U53 * 10


def test_rerun_bitwise_deterministic(gpu):
    """No atomics or races in the sweep: a rerun gives identical bits."""
    case = inputs.spheres_shock_3d(shape=(40, 32, 24), seed=4, nsph=5, rmin_cells=3, rmax_cells=7)
    go, g = grids(case)
    U0 = oracle.prim_to_cons(go, case.V)
    outs = []
    for _ in range(2):
        U = to_dev(U0)
        g.bind(U)
        g.rk_step(cfl=0.2, nsteps=3)
        outs.append(U.clone())
    assert torch.equal(outs[0], outs[1])


def test_status_reports_inadmissible_state(gpu):
    """A state with zero density (injected on the host) is reported through the
    device status word, not by a trap."""
    c = inputs.interface_advection_1d(n=64)
    go, g = grids(c)
    U = oracle.prim_to_cons(go, c.V)
    U[0:2, 10] = 0.0
    Ud = to_dev(U)
    g.bind(Ud)
    g.rk_step(cfl=0.5)
    with pytest.raises(wenoc.WcError) as ei:
        g.sync_status()
    assert ei.value.status in (3, 4)
    g.sync_status()  # cleared


@pytest.mark.parametrize("kind", ["negative_mass", "fraction_above_one", "sum", "psi", "nan"])
def test_check_state_admissible_set(gpu, kind):
    """wc_check_state against Eq. 8 on a state injected on the host: the
    clean state passes, one spoiled cell is reported (count 1, its index)."""
    c = inputs.shock_bubble_2d(nx=64, ny=32, seed=2)
    go, g = grids(c)
    U = oracle.prim_to_cons(go, c.V)
    Ud = to_dev(U)
    g.bind(Ud, validate=True)
    assert g.check_state(Ud) == (0, -1)
    N, d = c.N, c.dim
    cell = 17 * 64 + 11
    V = U.reshape(U.shape[0], -1).copy()
    if kind == "negative_mass":
        V[0, cell] = -1e-3
    elif kind == "fraction_above_one":
        V[N + d + 1, cell] = 1.0 + 1e-9
        V[N + d + 2, cell] = -1e-9
    elif kind == "sum":
        V[N + d + 1, cell] += 1e-6
    elif kind == "psi":
        V[N + d, cell] = 0.0          # rho E = 0: far below the energy bound
    else:
        V[N, cell] = np.nan
    Vd = to_dev(V.reshape(U.shape))
    with pytest.raises(wenoc.WcError) as ei:
        g.check_state(Vd)
    assert ei.value.status == 3
    nb, first = ctypes_check(g, Vd)
    assert nb == 1 and first == cell


def ctypes_check(g, U):
    import ctypes
    nb, first = ctypes.c_long(0), ctypes.c_long(0)
    rc = wenoc.lib().wc_check_state(g.h, ctypes.c_void_p(U.data_ptr()), 1e-10,
                                    ctypes.byref(nb), ctypes.byref(first), None)
    assert rc == 3
    return nb.value, first.value
