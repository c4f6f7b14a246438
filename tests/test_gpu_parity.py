"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

FP64 mode tolerance 1e-12 relative:
 * states after Runge-Kutta steps: max |U - U_or| over the grid relative to
   the largest |U_or| of the variable's group (each mass, the momentum
   vector, the energy, each fraction);
 * dU/dt: the change over one CFL-1 time step, max |L - L_or| / max_rate,
   relative to the same group scale.  (dU/dt itself is a difference of
   nearly equal fluxes; transverse momentum derivatives are pure round-off
   noise in these cases, so a per-variable max-|L| scale is meaningless.)
The inputs are identical bytes on both sides (the oracle's conservative map
of the seeded primitive state).
"""
import numpy as np
import pytest

import oracle
from paper_2608_00746_b300 import inputs

from gpu_util import SMALL_CASES, grids, rel_err_per_var, rhs_err, state_err, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("name", sorted(SMALL_CASES))
def test_rhs_parity_fp64(gpu, name):
    case = SMALL_CASES[name]()
    go, gg = grids(case)
    U = oracle.prim_to_cons(go, case.V)
    L_or = oracle.rhs(go, U)
    Ud = to_dev(U)
    gg.bind(Ud)
    L = gg.rhs(Ud).cpu().numpy()
    gg.sync_status()
    err = rhs_err(L, L_or, U, oracle.max_rate(go, U), case.N, case.dim)
    assert (err <= TOL).all(), (name, err)


@pytest.mark.parametrize("flux", ["hll", "hllc"])
def test_rhs_parity_both_fluxes_3d(gpu, flux):
    case = SMALL_CASES["spheres_3d_ragged"]()
    go, gg = grids(case, flux=flux)
    U = oracle.prim_to_cons(go, case.V)
    L_or = oracle.rhs(go, U)
    Ud = to_dev(U)
    gg.bind(Ud)
    err = rhs_err(gg.rhs(Ud).cpu().numpy(), L_or, U, oracle.max_rate(go, U), case.N, case.dim)
    assert (err <= TOL).all(), err


@pytest.mark.parametrize("name", ["slab_1d_hllc", "shock_bubble_2d_ragged", "spheres_3d_ragged"])
def test_rk3_parity_fp64(gpu, name):
    case = SMALL_CASES[name]()
    go, gg = grids(case)
    U = oracle.prim_to_cons(go, case.V)
    Ud = to_dev(U)
    gg.bind(Ud)
    cfl = case.cfl or 0.2
    for step in range(5):
        U, dt_or = oracle.rk3_step(go, U, cfl=cfl)
        dt = gg.rk_step(cfl=cfl, want_dt=True)
        assert dt == pytest.approx(dt_or, rel=1e-13)
        err = state_err(Ud.cpu().numpy(), U, case.N, case.dim)
        assert (err <= TOL).all(), (step, err)
    gg.sync_status()


def test_prim_cons_parity(gpu):
    case = SMALL_CASES["spheres_3d_ragged"]()
    go, gg = grids(case)
    V = case.V
    U_or = oracle.prim_to_cons(go, V)
    U = gg.prim_to_cons(to_dev(V)).cpu().numpy()
    assert (rel_err_per_var(U, U_or) <= 1e-15).all()
    V_or = oracle.cons_to_prim(go, U_or)
    V2 = gg.cons_to_prim(to_dev(U_or)).cpu().numpy()
    assert (rel_err_per_var(V2, V_or) <= 1e-12).all()


@pytest.mark.parametrize("N,seed", [(2, 0), (3, 1), (5, 2)])
def test_limit_parity(gpu, N, seed):
    """wc_limit (Eq. 17-21 alone) on adversarial raw faces vs the oracle.
    Cells where every fraction of a face is limited to zero (S = 0 in exact
    arithmetic, the oracle's first-order fallback, theta_17 = 0) sit on a
    rounding knife edge and are compared separately below."""
    d = 2
    Vb, VL, VR = inputs.random_admissible_stencils(3001, N, d, seed=seed)
    rng = np.random.default_rng(seed)
    gam = list(rng.uniform(1.2, 6.0, size=N))
    pinf = list(np.where(rng.uniform(size=N) < 0.5, 0.0, 10.0 ** rng.uniform(3, 8, size=N)))
    go = oracle.Grid((8, 8), (1.0, 1.0), gam, pinf)
    from paper_2608_00746_b300 import wenoc
    gg = wenoc.Grid((8, 8), (1.0, 1.0), gam, pinf)
    Ub = oracle.prim_to_cons(go, Vb)
    keep = oracle.psi(go, Ub) > 0
    Ub, VL, VR = (np.ascontiguousarray(a[:, keep]) for a in (Ub, VL, VR))
    UL_or, UR_or, TH_or = oracle.limit(go, Ub, VL, VR)
    UL, UR, TH = gg.limit(0, to_dev(Ub), to_dev(VL), to_dev(VR))
    UL, UR, TH = UL.cpu().numpy(), UR.cpu().numpy(), TH.cpu().numpy()
    # knife edge: a face sum S that is zero in exact arithmetic (either side
    # took the fallback, or normalised by a rounding-level S)
    ok = (TH_or[0] > 0) & (TH[0] > 0) & (TH_or[1] > 1e-8) & (TH[1] > 1e-8)
    assert ok.mean() > 0.9
    d = 2
    for A, B in ((UL, UL_or), (UR, UR_or)):
        err = state_err(A[:, ok], B[:, ok], N, d)
        assert (err <= 1e-12).all(), err
    # theta = fbar/(fbar - m) amplifies rounding of m when fbar - m is small
    assert np.abs(TH - TH_or)[:, ok].max() <= 1e-9
    # Eq. 8 at every limited face, knife-edge cells included, with no slack:
    # masses >= 0, fractions in [0, 1], unity sum to 2N 2^-53
    for A in (UL, UR):
        a = A[N + d + 1:]
        s = a[0].copy()
        for p in range(1, N):
            s = s + a[p]
        assert A[:N].min() >= 0.0 and a.min() >= 0.0 and a.max() <= 1.0
        assert np.abs(s - 1.0).max() <= 2 * N * 2.0 ** -53


def test_limit_degenerate_face_exact(gpu):
    """Both fractions of the left face limited exactly to zero (S = 0): the
    cell keeps its averages for masses and fractions (first-order fallback).
    The numbers are exact in binary so both implementations take the branch."""
    from paper_2608_00746_b300 import wenoc
    go = oracle.Grid((8,), (1.0,), [1.4, 1.4], [0.0, 0.0])
    gg = wenoc.Grid((8,), (1.0,), [1.4, 1.4], [0.0, 0.0])
    # averages alpha = (0.5, 0.5); raw left faces -0.5 each, right faces 0.5
    Vb = np.array([[0.5], [0.5], [0.0], [1.0], [0.5], [0.5]])
    VL = np.array([[-0.5], [-0.5], [0.0], [1.0], [-0.5], [-0.5]])
    VR = np.array([[0.5], [0.5], [0.0], [1.0], [0.5], [0.5]])
    Ub = oracle.prim_to_cons(go, Vb)
    UL_or, UR_or, TH_or = oracle.limit(go, Ub, VL, VR)
    UL, UR, TH = gg.limit(0, to_dev(Ub), to_dev(VL), to_dev(VR))
    assert TH_or[0, 0] == 0.0 and TH.cpu().numpy()[0, 0] == 0.0
    for A, B in ((UL.cpu().numpy(), UL_or), (UR.cpu().numpy(), UR_or)):
        assert np.allclose(A, B, rtol=1e-14, atol=1e-14)
        assert np.allclose(B[[0, 1, 4, 5]], Ub[[0, 1, 4, 5]], rtol=1e-15)


@pytest.mark.parametrize("seg", [5, 14])
@pytest.mark.parametrize("name", ["slab_1d_hllc", "shock_bubble_2d_ragged", "spheres_3d_ragged"])
def test_rhs_parity_segment_schedule(gpu, name, seg):
    """The per-thread segment march (seg > 0; the batched patches use it) is
    held to the same tolerance as the default window schedule."""
    case = SMALL_CASES[name]()
    go, gg = grids(case, seg=seg)
    U = oracle.prim_to_cons(go, case.V)
    L_or = oracle.rhs(go, U)
    Ud = to_dev(U)
    gg.bind(Ud)
    L = gg.rhs(Ud).cpu().numpy()
    gg.sync_status()
    err = rhs_err(L, L_or, U, oracle.max_rate(go, U), case.N, case.dim)
    assert (err <= TOL).all(), (name, seg, err)


@pytest.mark.parametrize("block", [32, 64, 128])
@pytest.mark.parametrize("name", ["shock_bubble_2d_ragged", "spheres_3d_ragged"])
def test_rhs_parity_window_block_sizes(gpu, name, block):
    """The window sweep gives the same dU/dt whatever the warps per block
    (each warp takes whole windows; the block size only changes residency)."""
    case = SMALL_CASES[name]()
    go, gg = grids(case, block=block)
    U = oracle.prim_to_cons(go, case.V)
    L_or = oracle.rhs(go, U)
    Ud = to_dev(U)
    gg.bind(Ud)
    L = gg.rhs(Ud).cpu().numpy()
    gg.sync_status()
    err = rhs_err(L, L_or, U, oracle.max_rate(go, U), case.N, case.dim)
    assert (err <= TOL).all(), (name, block, err)


@pytest.mark.parametrize("shape", [(91, 8), (64, 31), (62, 40), (33, 17)])
def test_rhs_parity_window_tails(gpu, shape):
    """Pencils whose last cells are taken several pencils to a warp (tails of
    1, 2, 3, 4, 8 and 10 cells, a partly filled last warp, lanes past the
    last group) and short reflective pencils (8 and 17 cells) whose window
    lanes run past the ghost layers: dU/dt and three Runge-Kutta steps."""
    case = inputs.shock_bubble_2d(nx=shape[0], ny=shape[1], seed=5)
    go, gg = grids(case)
    U = oracle.prim_to_cons(go, case.V)
    Ud = to_dev(U)
    gg.bind(Ud)
    L = gg.rhs(Ud).cpu().numpy()
    gg.sync_status()
    err = rhs_err(L, oracle.rhs(go, U), U, oracle.max_rate(go, U), case.N, case.dim)
    assert (err <= TOL).all(), (shape, err)
    for _ in range(3):
        U, dt = oracle.rk3_step(go, U, cfl=0.2)
        gg.rk_step(dt=dt)
    gg.sync_status()
    err = state_err(Ud.cpu().numpy(), U, case.N, case.dim)
    assert (err <= TOL).all(), (shape, err)


@pytest.mark.parametrize("precision", ["mixed", "learned"])
@pytest.mark.parametrize("name", ["shock_bubble_2d_ragged", "spheres_3d_ragged", "circles_2d_n3",
                                  "slab_1d_hllc", "five_phase_2d"])
def test_split_sweep_equals_single_pass(gpu, name, precision):
    """The reduced precisions' split sweep (face pass into the workspace's
    face buffer, then the flux pass) and the single-pass sweep (a workspace
    without the face buffer) give the same rhs and steps bit for bit."""
    import torch
    from paper_2608_00746_b300 import surrogate, wenoc
    case = SMALL_CASES[name]()
    if precision == "learned" and case.N > 3:
        pytest.skip("the surrogate takes N <= 3")
    outs = []
    for faces in (True, False):
        go, g = grids(case, precision=precision)
        if precision == "learned":
            g.set_mlp(surrogate.Surrogate(seed=5).params, tau=1.0)
        U = to_dev(oracle.prim_to_cons(go, case.V))
        g.bind(U, g.new_workspace(faces=faces))
        L = g.rhs(U).clone()
        g.rk_step(cfl=case.cfl or 0.2, nsteps=5)
        g.sync_status()
        outs.append((L, U))
    assert wenoc.lib().wc_face_buffer_bytes(g.h) > 0
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("variant", ["fp64", "mixed", "learned", "weno_w", "cl_kapila"])
@pytest.mark.parametrize("name", ["shock_bubble_2d_ragged", "spheres_3d_ragged", "circles_2d_n3",
                                  "slab_1d_hllc", "five_phase_2d"])
def test_primitive_slots_equal_sweep_conversion(gpu, name, variant):
    """The primitive slots of a stage's input (one conversion pass whose
    slots the direction sweeps copy; mirrored boundary images still
    converted in the sweep) against sweeps that convert their cells
    themselves (a workspace without the slots): the rhs, the Phase-Field rhs
    and Runge-Kutta steps bit for bit, in every precision, the comparison
    scheme and WENO-CL with the Kapila model; the CFL time step taken in the
    first stage's slot pass equals k_max_rate's bit for bit."""
    import torch
    from paper_2608_00746_b300 import surrogate, wenoc
    case = SMALL_CASES[name]()
    precision = variant if variant in ("fp64", "mixed", "learned") else "fp64"
    kw = {"weno_w": {"scheme": "w"}, "cl_kapila": {"scheme": "cl", "kmodel": "kapila"}}.get(
        variant, {})
    if precision == "learned" and case.N > 3:
        pytest.skip("the surrogate takes N <= 3")
    outs = []
    for prim in (True, False):
        go, g = grids(case, precision=precision, **kw)
        if precision == "learned":
            g.set_mlp(surrogate.Surrogate(seed=5).params, tau=1.0)
        U = to_dev(oracle.prim_to_cons(go, case.V))
        g.bind(U, g.new_workspace(faces=False, prim=prim))
        L = g.rhs(U).clone()
        Q = to_dev(np.random.default_rng(3).normal(size=(case.N,) + tuple(U.shape[1:])) * 0.05)
        Lpf = g.rhs_pf(U, Q, dt_limit=2e-3).clone()
        # (CFL steps: with the slots the first stage's slot pass also takes
        # the rate, otherwise k_max_rate does)
        dt = g.rk_step(cfl=case.cfl or 0.2, nsteps=3, want_dt=True)
        try:  # (the unlimited comparison scheme may fail at a shock: alike in both)
            g.sync_status()
            status = "ok"
        except wenoc.WcError as e:
            status = str(e)
        outs.append((L, Lpf, U, status, dt))
    assert (wenoc.lib().wc_prim_buffer_bytes(g.h) > 0) == (case.dim > 1)
    assert outs[0][3] == outs[1][3]
    assert outs[0][4] == outs[1][4] or outs[0][3] != "ok"
    if variant != "weno_w":
        assert outs[0][3] == "ok"
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a.view(torch.int64), b.view(torch.int64))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "learned"])
@pytest.mark.parametrize("name", ["shock_bubble_2d_ragged", "spheres_3d_ragged", "circles_2d_n3",
                                  "slab_1d_hllc", "five_phase_2d"])
def test_host_buffer_step_equals_device_step(gpu, name, precision):
    """wc_rk_step_host (the upload overlapping the first sweep in bands of
    rows, the download overlapping the last sweep in bands of pencils; 1-D
    and the learned precision in sequence) gives the device step's states
    bit for bit: in place over several CFL steps, and into a second host
    buffer with a fixed time step."""
    import torch
    from paper_2608_00746_b300 import surrogate
    case = SMALL_CASES[name]()
    if precision == "learned" and case.N > 3:
        pytest.skip("the surrogate takes N <= 3")
    go, g = grids(case, precision=precision)
    if precision == "learned":
        g.set_mlp(surrogate.Surrogate(seed=5).params, tau=1.0)
    U0 = oracle.prim_to_cons(go, case.V)
    cfl = case.cfl or 0.2
    dt = 0.3 / oracle.max_rate(go, U0)
    for kw, nsteps, inplace in (({"cfl": cfl}, 3, True), ({"dt": dt}, 1, False)):
        Ud = to_dev(U0)
        g.bind(Ud)
        g.rk_step(nsteps=nsteps, **kw)
        torch.cuda.synchronize()
        g.sync_status()
        ref = Ud.cpu().reshape(-1)
        h_in = torch.from_numpy(U0.copy()).reshape(-1).pin_memory()
        h_out = h_in if inplace else torch.full_like(h_in, float("nan")).pin_memory()
        Ub = torch.full_like(Ud, float("nan"))  # the upload fills the bound state
        g.bind(Ub)
        g.rk_step_host(h_in, h_out, nsteps=nsteps, **kw)
        torch.cuda.synchronize()
        g.sync_status()
        assert torch.equal(h_out, ref), (kw, nsteps)
        assert torch.equal(Ub.cpu().reshape(-1), ref)
        if not inplace:
            assert torch.equal(h_in, torch.from_numpy(U0.copy()).reshape(-1))
