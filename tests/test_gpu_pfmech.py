"""The Phase-Field mechanism of the time step on the GPU (Eq. 28, Eq. 4 and
the Phase-Field step Eq. 5; reading R17) against the oracle: [div J_p]^ to
1e-12, the Q-map's solution checked with the oracle's operator and against
the oracle's face fluxes, the Phase-Field step to 1e-12 with a common Q,
full time steps to the Q-map's tolerance, and the invariants of long runs
(conservation, fraction sum, bounds, the equilibrium interface band)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import pf
from paper_2608_00746_b300 import inputs, wenoc

from gpu_util import SMALL_CASES, l1_group, state_err, to_dev

pytestmark = pytest.mark.gpu


def _grids(case):
    go = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                     bc=case.bc)
    g = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                   bc=case.bc)
    return go, g


CASES = {
    "two_phase_advection": lambda: inputs.two_phase_advection_2d(n=40),
    "five_phase_2d": SMALL_CASES["five_phase_2d"],
    "shock_bubble_2d_ragged": SMALL_CASES["shock_bubble_2d_ragged"],
    "spheres_3d_ragged": SMALL_CASES["spheres_3d_ragged"],
    "slab_1d_hllc": SMALL_CASES["slab_1d_hllc"],
}


def _evolved(name, steps=3):
    case = CASES[name]()
    go, g = _grids(case)
    U = oracle.prim_to_cons(go, case.V)
    dt = case.meta.get("dt") if case.meta else None
    for _ in range(steps):
        U, _ = oracle.rk3_step(go, U, cfl=case.cfl or 0.2, dt=dt or 0.0)
    return case, go, g, U


@pytest.mark.parametrize("name", sorted(CASES))
def test_cac_rhs_parity(gpu, name):
    case, go, g, U = _evolved(name)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    R = g.cac_rhs(Ud).cpu().numpy()
    R_or, B_or, M_or = pf.cac_rhs(go, U)
    scale = max(np.abs(R_or).max(), M_or / case.dx[0] ** 2 * 1e-3)
    assert np.abs(R - R_or).max() <= 1e-12 * scale, (np.abs(R - R_or).max(), scale)
    # a given mobility is used as given
    R1 = g.cac_rhs(Ud, M=1.0).cpu().numpy()
    R1_or, _, _ = pf.cac_rhs(go, U, M=1.0)
    assert np.abs(R1 - R1_or).max() <= 1e-12 * np.abs(R1_or).max()


def _face_flux(go, phi, Q):
    """c_f (Q_b - Q_a)/dx on every coupled face, per phase and direction."""
    out = []
    for p in range(go.N):
        for d, (cf, a, b) in enumerate(pf.face_coefficients(go, phi[p])):
            q = Q[p].reshape(-1)
            on = cf > 0.0
            out.append(cf[on] * (q[b[on]] - q[a[on]]) / go.dx[d])
    return np.concatenate(out)


@pytest.mark.parametrize("name", ["two_phase_advection", "five_phase_2d",
                                  "shock_bubble_2d_ragged", "spheres_3d_ragged"])
def test_qmap_solution(gpu, name):
    """The GPU's Q solves the oracle's discrete Eq. 4 (the region-consistent
    right-hand side) to the requested tolerance, and its face fluxes
    c_f grad Q agree with the oracle's exact solution."""
    case, go, g, U = _evolved(name, steps=5)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    R = g.cac_rhs(Ud)
    Q, iters, res = g.qmap(Ud, tol=1e-13)
    assert res <= 1e-13 and iters > 0
    Q = Q.cpu().numpy()
    phi = pf.fractions(go, U)
    R_or, _, _ = pf.cac_rhs(go, U)
    Q_or, Rp = pf.qmap(go, phi, R_or)
    for p in range(go.N):
        A, _ = pf.qmap_operator(go, phi[p])
        AQ = A @ Q[p].reshape(-1)
        assert np.abs(AQ - Rp[p].reshape(-1)).max() <= 1e-9 * max(np.abs(R_or).max(), 1e-300)
    F, F_or = _face_flux(go, phi, Q), _face_flux(go, phi, Q_or)
    assert np.abs(F - F_or).max() <= 1e-8 * max(np.abs(F_or).max(), 1e-300)


def test_qmap_trace_fraction_next_to_zero(gpu):
    """A cell holding a trace fraction (the smallest denormal, below 2^-52:
    coefficient 0 by R17) beside cells with phi = 0, while its neighbour
    belongs to the interface band through its other face: Eq. 4 couples it
    to nothing.  The region labelling follows the operator's face weights
    (it never reads the label of a cell off the band); Q solves the
    oracle's Eq. 4 and is 0 at the trace cell."""
    case = inputs.interface_advection_1d(n=200)
    go, g = _grids(case)
    U = oracle.prim_to_cons(go, case.V)
    a0 = case.N + case.dim + 1
    air = U[a0]
    k = int(np.flatnonzero(air > 0.0)[0])      # first cell of the slab's band
    i = k - 2                                   # two cells outside it
    assert air[i - 1] == 0.0 and air[i] == 0.0 and air[i + 1] == 0.0
    tiny = np.nextafter(0.0, 1.0)               # 4.9e-324
    U[a0, i] = tiny
    U[a0 + 1, i] = 1.0 - tiny                   # = 1.0
    U[0, i] = tiny                              # the air mass (rho_air = 1)
    phi = pf.fractions(go, U)
    c = pf.coefficient(phi)
    assert phi[0, i] == tiny and c[0, i] == 0.0 and c[0, i + 1] == 0.0 and c[0, k] > 0.0
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    g.cac_rhs(Ud)
    Q, iters, res = g.qmap(Ud, tol=1e-13)
    assert res <= 1e-13
    Q = Q.cpu().numpy()
    R_or, _, _ = pf.cac_rhs(go, U)
    Q_or, Rp = pf.qmap(go, phi, R_or)
    for p in range(go.N):
        A, _ = pf.qmap_operator(go, phi[p])
        AQ = A @ Q[p].reshape(-1)
        assert np.abs(AQ - Rp[p].reshape(-1)).max() <= 1e-9 * max(np.abs(R_or).max(), 1e-300)
    assert Q[0, i] == 0.0  # a cell that no face couples keeps Q = 0
    F, F_or = _face_flux(go, phi, Q), _face_flux(go, phi, Q_or)
    assert np.abs(F - F_or).max() <= 1e-8 * max(np.abs(F_or).max(), 1e-300)


def test_qmap_warm_start(gpu):
    """Started from its own solution the Q-map does no iteration and keeps
    Q; started from that solution plus noise of size 1e-6 it converges to
    the same face fluxes in fewer iterations than from zero."""
    case, go, g, U = _evolved("shock_bubble_2d_ragged", steps=5)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    g.cac_rhs(Ud)
    Q, it0, _ = g.qmap(Ud, tol=1e-12)
    Q1 = Q.clone()
    _, it1, res1 = g.qmap(Ud, Q=Q1, tol=1e-12, warm=True)
    assert it1 == 0 and res1 <= 1e-12 and torch.equal(Q1, Q)
    rng = np.random.default_rng(3)
    Q2 = Q + to_dev(rng.normal(size=Q.shape) * 1e-6)
    _, it2, res2 = g.qmap(Ud, Q=Q2, tol=1e-12, warm=True)
    assert res2 <= 1e-12 and it2 < it0, (it0, it2, res2)
    phi = pf.fractions(go, U)
    F, F2 = _face_flux(go, phi, Q.cpu().numpy()), _face_flux(go, phi, Q2.cpu().numpy())
    assert np.abs(F - F2).max() <= 1e-8 * np.abs(F).max()


@pytest.mark.parametrize("qscale", [1.0, 1e4])
@pytest.mark.parametrize("name", ["two_phase_advection", "five_phase_2d", "spheres_3d_ragged"])
def test_pf_step_parity_with_common_q(gpu, name, qscale):
    """The Phase-Field step (SSP-RK3 of Eq. 5, gradients limited for dt) with
    the oracle's Q on both sides: 1e-12.  Q x 1e4 makes the gradient limit
    act on most coupled faces, in every direction's sweep."""
    case, go, g, U = _evolved(name)
    R_or, _, _ = pf.cac_rhs(go, U)
    Q, _ = pf.qmap(go, pf.fractions(go, U), R_or)
    Q = Q * qscale
    dt = 1e-3 if name == "two_phase_advection" else 0.5 * oracle.rk3_step(go, U, cfl=0.2)[1]
    Un = pf.pf_step(go, U, Q, dt)
    Ud = to_dev(U)
    g.bind(Ud)
    g.pf_step(to_dev(Q), dt)
    g.sync_status()
    err = state_err(Ud.cpu().numpy(), Un, case.N, case.dim)
    assert (err <= 1e-12).all(), err


def test_full_steps_match_oracle(gpu):
    """Ten time steps of Sec. 2.2 (hyperbolic, Eq. 28, Eq. 4, Phase-Field) on
    the Sec. 4.1.1 layout, 40^2: the states agree to the Q-map's accuracy."""
    case = inputs.two_phase_advection_2d(n=40)
    go, g = _grids(case)
    U = oracle.prim_to_cons(go, case.V)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    for _ in range(10):
        U, _, _ = pf.full_step(go, U, dt=case.meta["dt"])
        g.step(dt=case.meta["dt"], tol=1e-13)
    g.sync_status()
    err = state_err(Ud.cpu().numpy(), U, case.N, case.dim)
    assert (err <= 1e-9).all(), err


def test_full_steps_keep_invariants_and_the_equilibrium_band(gpu):
    """Sec. 4.1.1 air circle on the paper's 100^2 grid, one period (1000
    steps) with the mechanism: each phase's mass and fraction, momentum and
    energy conserved, fractions within rounding of [0, 1] summing to one, and
    the 0.05 < phi < 0.95 band at the equilibrium width (4.16 cells around
    the radius of 20 cells: 2 pi 20 x 4.16 = 523 cells)."""
    case = inputs.two_phase_advection_2d(n=100)
    go, g = _grids(case)
    Ud = to_dev(oracle.prim_to_cons(go, case.V))
    g.bind(Ud).set_pf_workspace(Ud.device)
    tot0 = Ud.sum(dim=(1, 2))
    g.step(dt=case.meta["dt"], nsteps=1000, tol=1e-10)
    g.sync_status()
    tot = Ud.sum(dim=(1, 2))
    scale = Ud.abs().sum(dim=(1, 2))
    assert ((tot - tot0).abs() <= 1e-11 * scale).all()
    a = Ud[5:7]
    assert a.min().item() >= -1e-10 and a.max().item() <= 1 + 1e-10
    assert (a.sum(0) - 1).abs().max().item() < 1e-12
    band = int(((a[0] > 0.05) & (a[0] < 0.95)).sum().item())
    expect = 2 * np.pi * 20 * 2 * np.sqrt(2) * np.arctanh(0.9)
    assert 0.85 * expect <= band <= 1.15 * expect, (band, expect)
    V = g.cons_to_prim(Ud).cpu().numpy()
    assert np.abs(V[2:4] - 1.0).max() < 1e-9


@pytest.mark.parametrize("n", [200, 300])
def test_qmap_solution_on_a_fully_mixed_grid(gpu, n):
    """Fractions inside (0, 1) on every cell of an n^2 periodic grid: one
    region of n^2 unknowns a phase.  40,000 (n = 200) take the
    register-resident iteration with two unknowns a thread (one a thread
    holds 148 x 256 = 37,888); 90,000 (n = 300) are more than two a thread
    and take the iteration on the lists in memory.  Either way Q solves the
    oracle's discrete Eq. 4."""
    case = inputs.two_phase_advection_2d(n=n)
    go, g = _grids(case)
    V = case.V.copy()
    ny, nx = V.shape[1:]
    yy, xx = np.meshgrid((np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx, indexing="ij")
    a1 = 0.5 + 0.3 * np.sin(2 * np.pi * xx) * np.sin(2 * np.pi * yy)
    rho = case.meta["rho"]
    V[0], V[1] = rho[0] * a1, rho[1] * (1 - a1)
    V[5], V[6] = a1, 1 - a1
    U = oracle.prim_to_cons(go, V)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    g.cac_rhs(Ud)
    Q, iters, res = g.qmap(Ud, tol=1e-12, maxit=20000)
    assert res <= 1e-12 and iters > 0
    flags = g.pfws.view(torch.int32)[-64:].cpu().numpy()
    assert list(flags[12:14]) == [n * n, n * n] and flags[17] == (2 if n == 200 else 0)
    Q = Q.cpu().numpy()
    phi = pf.fractions(go, U)
    R_or, _, _ = pf.cac_rhs(go, U)
    _, Rp = pf.qmap(go, phi, R_or)
    for p in range(go.N):
        A, _ = pf.qmap_operator(go, phi[p])
        AQ = A @ Q[p].reshape(-1)
        assert np.abs(AQ - Rp[p].reshape(-1)).max() <= 1e-8 * max(np.abs(R_or).max(), 1e-300)


def test_qmap_solution_three_phases_in_memory(gpu):
    """Three phases mixed on every cell of a 210^2 periodic grid (44,100
    unknowns a phase: more than one a thread, and N = 3 keeps at most one
    in registers), so the in-memory launch runs for N = 3; its Q solves the
    oracle's discrete Eq. 4 for every phase."""
    case = inputs.multiphase_advection_2d(n=210, nphase=3)
    go, g = _grids(case)
    V = case.V.copy()
    ny, nx = V.shape[1:]
    yy, xx = np.meshgrid((np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx, indexing="ij")
    a1 = 0.35 + 0.2 * np.sin(2 * np.pi * xx) * np.sin(2 * np.pi * yy)
    a2 = 0.3 + 0.15 * np.cos(2 * np.pi * xx)
    a = [a1, a2, 1.0 - a1 - a2]
    rho = [inputs.TABLE1[p][0] for p in range(3)]
    for p in range(3):
        V[p] = rho[p] * a[p]
        V[6 + p] = a[p]
    U = oracle.prim_to_cons(go, V)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    g.cac_rhs(Ud)
    Q, iters, res = g.qmap(Ud, tol=1e-12, maxit=20000)
    assert res <= 1e-12 and iters > 0
    band, per_thread = g.pf_band()
    assert band == [nx * ny] * 3 and per_thread == 0
    Q = Q.cpu().numpy()
    phi = pf.fractions(go, U)
    R_or, _, _ = pf.cac_rhs(go, U)
    _, Rp = pf.qmap(go, phi, R_or)
    for p in range(go.N):
        A, _ = pf.qmap_operator(go, phi[p])
        AQ = A @ Q[p].reshape(-1)
        assert np.abs(AQ - Rp[p].reshape(-1)).max() <= 1e-8 * max(np.abs(R_or).max(), 1e-300)


def test_qmap_and_full_step_without_an_interface(gpu):
    """A grid holding one pure phase (fractions exactly 0 and 1, no cell
    with phi (1 - phi) > 0): the band is empty, the Q-map does no
    iteration and returns Q = 0 (cold) or keeps the Q given (warm), and a
    full time step equals the hyperbolic step alone, bit for bit."""
    case = inputs.two_phase_advection_2d(n=40)
    go, g = _grids(case)
    V = case.V.copy()
    V[0], V[1], V[5], V[6] = 0.0, case.meta["rho"][1], 0.0, 1.0
    U = oracle.prim_to_cons(go, V)
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    g.cac_rhs(Ud)
    Q, iters, res = g.qmap(Ud, tol=1e-12)
    assert iters == 0 and g.pf_band() == ([0, 0], 1)
    assert not Q.any()
    Qw = torch.full_like(Q, 3.0)
    _, iters, _ = g.qmap(Ud, Q=Qw, tol=1e-12, warm=True)
    assert iters == 0 and bool((Qw == 3.0).all())
    U2 = Ud.clone()
    g2 = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                    bc=case.bc)
    g2.bind(U2)
    g.step(dt=case.meta["dt"])
    g2.rk_step(dt=case.meta["dt"])
    g.sync_status()
    g2.sync_status()
    assert torch.equal(Ud, U2)


@pytest.mark.parametrize("name", ["shock_bubble_2d_ragged", "spheres_3d_ragged", "in_memory"])
def test_qmap_and_full_steps_repeat_bit_for_bit(gpu, name):
    """The Q-map's region sums are order-independent and its reductions run
    in a fixed order, so Q (register-resident and in-memory iterations
    alike) and full time steps are the same bit for bit on every run."""
    if name == "in_memory":
        case = inputs.multiphase_advection_2d(n=210, nphase=3)
        go, g = _grids(case)
        V = case.V.copy()
        ny, nx = V.shape[1:]
        yy, xx = np.meshgrid((np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                             indexing="ij")
        a1 = 0.35 + 0.2 * np.sin(2 * np.pi * xx) * np.sin(2 * np.pi * yy)
        a2 = 0.3 + 0.15 * np.cos(2 * np.pi * xx)
        a = [a1, a2, 1.0 - a1 - a2]
        for p in range(3):
            V[p] = inputs.TABLE1[p][0] * a[p]
            V[6 + p] = a[p]
        U = oracle.prim_to_cons(go, V)
        dt = None
    else:
        case, go, g, U = _evolved(name, steps=5)
        dt = case.meta.get("dt") if case.meta else None
    Ud = to_dev(U)
    g.bind(Ud).set_pf_workspace(Ud.device)
    g.cac_rhs(Ud)
    runs = [g.qmap(Ud, tol=1e-12, maxit=20000) for _ in range(3)]
    if name == "in_memory":
        assert g.pf_band()[1] == 0
    for Q, iters, res in runs[1:]:
        assert iters == runs[0][1] and res == runs[0][2]
        assert torch.equal(Q, runs[0][0])
    if name == "in_memory":
        return
    # full steps start the Q-map from the grid's last Q: a fresh grid each
    outs = []
    for _ in range(2):
        _, g = _grids(case)
        Us = to_dev(U)
        g.bind(Us).set_pf_workspace(Us.device)
        if dt:
            g.step(dt=dt, nsteps=3)
        else:
            g.step(cfl=case.cfl or 0.2, nsteps=3)
        g.sync_status()
        outs.append(Us)
    assert torch.equal(outs[0], outs[1])


def test_full_steps_in_mixed_precision(gpu):
    """Full time steps with the mechanism in the mixed precision (the split
    sweep's face and flux passes for both the hyperbolic and the Phase-Field
    step, the Q-map in FP64): after ten steps of the ragged shock-bubble the
    state is within the L1 bound of the FP64 steps, masses >= 0 and fractions
    in [0, 1] exactly at cell averages, and their sum one to round-off."""
    case, go, g64, U = _evolved("shock_bubble_2d_ragged", steps=2)
    gm = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                    bc=case.bc, precision="mixed")
    A, B = to_dev(U), to_dev(U)
    g64.bind(A).set_pf_workspace(A.device)
    gm.bind(B).set_pf_workspace(B.device)
    N, d = case.N, case.dim
    for _ in range(10):
        dt = g64.rk_step(cfl=case.cfl, want_dt=True)
        g64.cac_rhs(A)
        Q, _, _ = g64.qmap(A, tol=1e-12)
        g64.pf_step(Q, dt)
        gm.step(dt=dt, nsteps=1, tol=1e-12)
    g64.sync_status()
    gm.sync_status()
    a, b = A.cpu().numpy(), B.cpu().numpy()
    assert (l1_group(b, a, N, d) <= 1e-5).all(), l1_group(b, a, N, d)
    assert b[:N].min() >= 0.0
    frac = b[N + d + 1:]
    assert frac.min() >= 0.0 and frac.max() <= 1.0
    # the sum's drift: at most 2N units of 2^-53 a step of each of the two
    # stepping stages (hyperbolic, Phase-Field), from the starting state's
    sum0 = np.abs(U[N + d + 1:].sum(0) - 1.0).max()
    assert np.abs(frac.sum(0) - 1.0).max() <= sum0 + 2 * 2 * N * 2.0 ** -53 * 10


def test_pf_step_with_quiet_windows(gpu):
    """A 515 x 247 shock-bubble whose interface band covers a part of the
    grid: windows where every face has G = 0 carry no Phase-Field flux and
    skip the reconstruction, limiter and flux.  With every workspace byte
    that a step does not write set to NaN first (stage buffers, accumulator,
    face buffer), the FP64 Phase-Field step matches the oracle to 1e-12, the
    mixed precision's split sweep (whose face pass writes no faces in such
    windows, and whose flux pass reads none where G = 0) equals its single
    pass bit for bit, within the L1 bound of the FP64 step, and no status
    bit is set."""
    case = inputs.shock_bubble_2d(nx=515, ny=247, seed=5)
    go, g64 = _grids(case)
    U = oracle.prim_to_cons(go, case.V)
    for _ in range(2):
        U, _ = oracle.rk3_step(go, U, cfl=case.cfl)
    R_or, _, _ = pf.cac_rhs(go, U)
    Q, _ = pf.qmap(go, pf.fractions(go, U), R_or)
    band = (Q != 0.0).any(0)
    assert 0.02 < band.mean() < 0.5, band.mean()
    dt = 0.5 * oracle.rk3_step(go, U, cfl=case.cfl)[1]
    Un = pf.pf_step(go, U, Q, dt)
    Qd = to_dev(Q)
    A = to_dev(U)
    ws = g64.new_workspace().fill_(float("nan"))
    g64.bind(A, ws)
    g64.pf_step(Qd, dt)
    g64.sync_status()
    a = A.cpu().numpy()
    err = state_err(a, Un, case.N, case.dim)
    assert (err <= 1e-12).all(), err
    assert not np.array_equal(a, U)
    outs = []
    for faces in (True, False):
        gm = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                        bc=case.bc, precision="mixed")
        B = to_dev(U)
        gm.bind(B, gm.new_workspace(faces=faces).fill_(float("nan")))
        gm.pf_step(Qd, dt)
        gm.sync_status()
        outs.append(B)
    assert torch.equal(outs[0], outs[1])
    b = outs[0].cpu().numpy()
    assert np.isfinite(b).all()
    assert (l1_group(b, a, case.N, case.dim) <= 1e-5).all(), l1_group(b, a, case.N, case.dim)
