"""Batched AMR-like patches (config-4 shape, reduced count): every patch
against the FP64 oracle run on that patch as its own grid (outflow
boundaries, cell size 1/edge), one persistent launch per stage, graph
capture, schedules and the autotuner."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_00746_b300 import inputs, wenoc

from gpu_util import l1_group, momentum_floor, rhs_err, state_err, to_dev

pytestmark = pytest.mark.gpu
N, D = 3, 3


def batch(npatch=24, seed=3):
    edges, states, (g, pi, Dm) = inputs.patch_batch(npatch=npatch, seed=seed)
    return [int(e) for e in edges], states, g, pi, Dm


def oracle_grid(e, g, pi, Dm):
    return oracle.Grid((e, e, e), (1.0 / e,) * 3, g, pi, Dm, flux="hll", bc=("outflow",) * 6)


def pooled_cons(P, edges, states, g, pi, Dm):
    Us = [oracle.prim_to_cons(oracle_grid(e, g, pi, Dm), S) for e, S in zip(edges, states)]
    return P.pack(Us), Us


def test_patch_rhs_parity_fp64(gpu):
    edges, states, g, pi, Dm = batch()
    assert set(edges) == {8, 12, 16, 24, 32} or len(set(edges)) >= 3
    P = wenoc.Patches(edges, g, pi, Dm, precision="fp64")
    U, Us = pooled_cons(P, edges, states, g, pi, Dm)
    Ud = to_dev(U)
    P.bind(Ud)
    L = P.rhs(Ud).cpu().numpy()
    P.sync_status()
    for p, e in enumerate(edges):
        go = oracle_grid(e, g, pi, Dm)
        L_or = oracle.rhs(go, Us[p])
        err = rhs_err(P.unpack(L, p), L_or, Us[p], oracle.max_rate(go, Us[p]), N, D,
                      mom_floor=momentum_floor(go, Us[p]))
        assert (err <= 1e-12).all(), (p, e, err)


def test_patch_rk_parity_fp64_graph_and_schedules(gpu):
    edges, states, g, pi, Dm = batch(npatch=16, seed=5)
    P = wenoc.Patches(edges, g, pi, Dm, precision="fp64")
    U, Us = pooled_cons(P, edges, states, g, pi, Dm)
    grids = [oracle_grid(e, g, pi, Dm) for e in edges]
    # global dt: cfl / max over patches of the CFL rate
    rate = max(oracle.max_rate(go, Up) for go, Up in zip(grids, Us))
    dt = 0.2 / rate
    outs = []
    s = torch.cuda.Stream()
    for sched, graph in [((64, 4, 1), False), ((128, 2, 0), False), ((64, 3, 1), True)]:
        Ud = to_dev(U)
        with torch.cuda.stream(s):
            P.bind(Ud, stream=s)
            P.set_schedule(*sched)
            P.rk_step(dt=dt, nsteps=2, use_graph=graph, stream=s)
        s.synchronize()
        P.sync_status(stream=s)
        outs.append(Ud.cpu().numpy())
    # the CFL time step computed on the device over all patches (first step)
    Uc = to_dev(U)
    with torch.cuda.stream(s):
        P.bind(Uc, stream=s)
        P.rk_step(cfl=0.2, nsteps=1, use_graph=True, stream=s)
    s.synchronize()
    U1 = Uc.cpu().numpy()
    for p, (go, Up) in enumerate(zip(grids, Us)):
        Uo, _ = oracle.rk3_step(go, Up, dt=dt)
        assert (state_err(P.unpack(U1, p), Uo, N, D, mom_floor=momentum_floor(go, Uo))
                <= 1e-12).all()
    # bit-identical whatever the schedule or the graph
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    for p, (go, Up) in enumerate(zip(grids, Us)):
        Uo = Up
        for _ in range(2):
            Uo, _ = oracle.rk3_step(go, Uo, dt=dt)
        err = state_err(P.unpack(outs[0], p), Uo, N, D, mom_floor=momentum_floor(go, Uo))
        assert (err <= 1e-12).all(), (p, err)


def test_patch_mixed_l1_and_bounds(gpu):
    edges, states, g, pi, Dm = batch(npatch=12, seed=7)
    P64 = wenoc.Patches(edges, g, pi, Dm, precision="fp64")
    Pmx = wenoc.Patches(edges, g, pi, Dm, precision="mixed")
    U, _ = pooled_cons(P64, edges, states, g, pi, Dm)
    A, B = to_dev(U), to_dev(U)
    P64.bind(A)
    Pmx.bind(B)
    for _ in range(5):
        P64.rk_step(dt=2e-7)
        Pmx.rk_step(dt=2e-7)
    torch.cuda.synchronize()
    P64.sync_status()
    Pmx.sync_status()
    a, b = A.cpu().numpy(), B.cpu().numpy()
    assert (l1_group(b, a, N, D) <= 1e-5).all()
    frac = b[N + D + 1:]
    assert frac.min() >= -4 * 2.0 ** -52 and frac.max() <= 1 + 4 * 2.0 ** -52


def test_patch_autotune_restores_state(gpu):
    edges, states, g, pi, Dm = batch(npatch=40, seed=9)
    P = wenoc.Patches(edges, g, pi, Dm, precision="mixed")
    U, _ = pooled_cons(P, edges, states, g, pi, Dm)
    Ud = to_dev(U)
    P.bind(Ud)
    best = P.autotune(cfl=0.2, steps=1)
    assert best["block"] in (64, 128) and best["ctas_per_sm"] in (2, 3, 4, 6)
    assert best["dynamic"] in (0, 1, 2)
    assert best["ms_per_step"] > 0
    assert np.array_equal(Ud.cpu().numpy(), U)


def test_patch_kapila_parity(gpu):
    """K_p of the Kapila model (Eq. 2-3, Wood's mixture speed) on every patch:
    rhs and one SSP-RK3 step against the oracle run with the same model, FP64;
    the mixed form within the L1 bound of the Allaire patches; a model outside
    the two is refused at setup."""
    edges, states, g, pi, Dm = batch(npatch=12, seed=11)

    def ogrid(e):
        return oracle.Grid((e, e, e), (1.0 / e,) * 3, g, pi, Dm, flux="hll",
                           bc=("outflow",) * 6, kmodel="kapila")

    P = wenoc.Patches(edges, g, pi, Dm, precision="fp64", kmodel="kapila")
    grids = [ogrid(e) for e in edges]
    Us = [oracle.prim_to_cons(go, S) for go, S in zip(grids, states)]
    U = P.pack(Us)
    Ud = to_dev(U)
    P.bind(Ud)
    L = P.rhs(Ud).cpu().numpy()
    P.sync_status()
    for p, (go, Up) in enumerate(zip(grids, Us)):
        err = rhs_err(P.unpack(L, p), oracle.rhs(go, Up), Up, oracle.max_rate(go, Up), N, D,
                      mom_floor=momentum_floor(go, Up))
        assert (err <= 1e-12).all(), (p, edges[p], err)
    # the CFL rate of the Kapila model differs from the Allaire one on mixed cells
    rate = max(oracle.max_rate(go, Up) for go, Up in zip(grids, Us))
    dt = 0.2 / rate
    P.rk_step(dt=dt)
    torch.cuda.synchronize()
    P.sync_status()
    U1 = Ud.cpu().numpy()
    for p, (go, Up) in enumerate(zip(grids, Us)):
        Uo, _ = oracle.rk3_step(go, Up, dt=dt)
        err = state_err(P.unpack(U1, p), Uo, N, D, mom_floor=momentum_floor(go, Uo))
        assert (err <= 1e-12).all(), (p, err)
    # the device CFL step uses Wood's speed: one step at cfl=0.2 matches the
    # oracle step at the oracle's Kapila dt
    Uc = to_dev(U)
    P.bind(Uc)
    P.rk_step(cfl=0.2)
    torch.cuda.synchronize()
    P.sync_status()
    U2 = Uc.cpu().numpy()
    for p, (go, Up) in enumerate(zip(grids, Us)):
        Uo, _ = oracle.rk3_step(go, Up, dt=dt)
        assert (state_err(P.unpack(U2, p), Uo, N, D, mom_floor=momentum_floor(go, Uo))
                <= 1e-12).all(), p
    Pm = wenoc.Patches(edges, g, pi, Dm, precision="mixed", kmodel="kapila")
    Um = to_dev(U)
    Pm.bind(Um)
    Pm.rk_step(dt=dt)
    torch.cuda.synchronize()
    Pm.sync_status()
    assert (l1_group(Um.cpu().numpy(), U1, N, D) <= 1e-5).all()
    with pytest.raises(KeyError):
        wenoc.Patches(edges, g, pi, Dm, kmodel="stiffened")


# edges for every window plan: groups of tails (3, 8, 31, 33), one tail a
# warp (15, 24), a full window and no tail (30), a window and a tail (32)
WIN_EDGES = (3, 8, 15, 24, 30, 31, 32, 33)


def test_patch_window_schedule_fp64_parity(gpu):
    """The window schedule (kind 2: per direction, the grids' window sweep
    over the pencils of each group of equal patches) against the oracle on
    every patch: rhs, an SSP-RK3 step at a given dt and at the device's CFL
    dt, at 1e-12; direct launches, graph replay, two block shapes and a
    workspace without the primitive slots bit for bit the same."""
    edges, states, (g, pi, Dm) = inputs.patch_batch(npatch=24, seed=17, edges=WIN_EDGES)
    edges = [int(e) for e in edges]
    assert set(edges) == set(WIN_EDGES)
    P = wenoc.Patches(edges, g, pi, Dm, precision="fp64")
    U, Us = pooled_cons(P, edges, states, g, pi, Dm)
    grids = [oracle_grid(e, g, pi, Dm) for e in edges]
    Ud = to_dev(U)
    P.bind(Ud)
    P.set_schedule(128, 3, 2)
    L = P.rhs(Ud).cpu().numpy()
    P.sync_status()
    for p, (go, Up) in enumerate(zip(grids, Us)):
        err = rhs_err(P.unpack(L, p), oracle.rhs(go, Up), Up, oracle.max_rate(go, Up), N, D,
                      mom_floor=momentum_floor(go, Up))
        assert (err <= 1e-12).all(), (p, edges[p], err)
    rate = max(oracle.max_rate(go, Up) for go, Up in zip(grids, Us))
    dt = 0.2 / rate
    outs = []
    s = torch.cuda.Stream()
    for sched, graph, kw, prim in [((128, 3, 2), False, {"dt": dt}, True),
                                   ((64, 4, 2), False, {"dt": dt}, True),
                                   ((128, 2, 2), True, {"dt": dt}, True),
                                   ((128, 3, 2), True, {"cfl": 0.2}, True),
                                   ((128, 3, 2), False, {"dt": dt}, False)]:
        Uw = to_dev(U)
        with torch.cuda.stream(s):
            P.bind(Uw, stream=s, faces=prim, prim=prim)
            P.set_schedule(*sched)
            P.rk_step(nsteps=1, use_graph=graph, stream=s, **kw)
        s.synchronize()
        P.sync_status(stream=s)
        outs.append(Uw.cpu().numpy())
    for k in (1, 2, 4):
        assert np.array_equal(outs[0], outs[k]), k
    for U1 in (outs[0], outs[3]):
        for p, (go, Up) in enumerate(zip(grids, Us)):
            Uo, _ = oracle.rk3_step(go, Up, dt=dt)
            err = state_err(P.unpack(U1, p), Uo, N, D, mom_floor=momentum_floor(go, Uo))
            assert (err <= 1e-12).all(), (p, edges[p], err)


def test_patch_window_schedule_mixed(gpu):
    """Mixed precision on the window schedule: the split sweep (face buffer in
    the workspace), the one-pass sweep (workspace without it) and the
    one-pass sweep converting its cells itself (no primitive slots either)
    give the same bits; five steps stay within the L1 bound of the FP64 patches with
    masses >= 0 and fractions in [0, 1] (exactly, at cell averages); the
    persistent schedule's mixed sweep meets the same bound."""
    edges, states, (g, pi, Dm) = inputs.patch_batch(npatch=16, seed=19, edges=WIN_EDGES)
    edges = [int(e) for e in edges]
    P64 = wenoc.Patches(edges, g, pi, Dm, precision="fp64")
    Pmx = wenoc.Patches(edges, g, pi, Dm, precision="mixed")
    assert wenoc.lib().wc_patches_face_buffer_bytes(P64.h) == 0
    assert wenoc.lib().wc_patches_face_buffer_bytes(Pmx.h) > 0
    U, _ = pooled_cons(P64, edges, states, g, pi, Dm)
    A = to_dev(U)
    P64.bind(A)
    outs = []
    for faces, prim in ((True, True), (False, True), (False, False)):
        B = to_dev(U)
        Pmx.bind(B, faces=faces, prim=prim)
        Pmx.set_schedule(128, 3, 2)
        for _ in range(5):
            Pmx.rk_step(dt=2e-7)
        torch.cuda.synchronize()
        Pmx.sync_status()
        outs.append(B.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    for _ in range(5):
        P64.rk_step(dt=2e-7)
    torch.cuda.synchronize()
    P64.sync_status()
    a, b = A.cpu().numpy(), outs[0]
    assert (l1_group(b, a, N, D) <= 1e-5).all()
    assert b[:N].min() >= 0.0
    frac = b[N + D + 1:]
    assert frac.min() >= 0.0 and frac.max() <= 1.0
    C = to_dev(U)
    Pmx.bind(C)
    Pmx.set_schedule(64, 4, 1)
    for _ in range(5):
        Pmx.rk_step(dt=2e-7)
    torch.cuda.synchronize()
    Pmx.sync_status()
    assert (l1_group(C.cpu().numpy(), a, N, D) <= 1e-5).all()


@pytest.mark.parametrize("flux", ["hll", "hllc"])
def test_patch_window_schedule_kapila_and_flux(gpu, flux):
    """The Kapila model with either flux in both schedule kinds (window
    sweeps and the persistent launch): rhs and an SSP-RK3 step of every patch
    against the oracle at 1e-12 (FP64)."""
    edges, states, (g, pi, Dm) = inputs.patch_batch(npatch=10, seed=29, edges=(8, 15, 24, 32))
    edges = [int(e) for e in edges]

    def ogrid(e):
        return oracle.Grid((e, e, e), (1.0 / e,) * 3, g, pi, Dm, flux=flux,
                           bc=("outflow",) * 6, kmodel="kapila")

    P = wenoc.Patches(edges, g, pi, Dm, flux=flux, precision="fp64", kmodel="kapila")
    grids = [ogrid(e) for e in edges]
    Us = [oracle.prim_to_cons(go, S) for go, S in zip(grids, states)]
    U = P.pack(Us)
    rate = max(oracle.max_rate(go, Up) for go, Up in zip(grids, Us))
    dt = 0.2 / rate
    for sched in [(128, 3, 2), (64, 4, 1)]:
        Ud = to_dev(U)
        P.bind(Ud)
        P.set_schedule(*sched)
        L = P.rhs(Ud).cpu().numpy()
        P.sync_status()
        for p, (go, Up) in enumerate(zip(grids, Us)):
            err = rhs_err(P.unpack(L, p), oracle.rhs(go, Up), Up, oracle.max_rate(go, Up), N, D,
                          mom_floor=momentum_floor(go, Up))
            assert (err <= 1e-12).all(), (sched, p, edges[p], err)
        P.rk_step(dt=dt)
        torch.cuda.synchronize()
        P.sync_status()
        U1 = Ud.cpu().numpy()
        for p, (go, Up) in enumerate(zip(grids, Us)):
            Uo, _ = oracle.rk3_step(go, Up, dt=dt)
            err = state_err(P.unpack(U1, p), Uo, N, D, mom_floor=momentum_floor(go, Uo))
            assert (err <= 1e-12).all(), (sched, p, err)
