"""Parity at the full workload sizes, in the launch configuration the
benchmark times (default window schedule, occupancy-sized persistent grid):
the FP64 operator against the FP64 oracle on whole grids -- the 2-D
shock-bubble (1024 x 512, N = 2), the 2-D circles (2048 x 2048, N = 3), the
3-D spheres (256^3, N = 3) -- after a few GPU steps (so limiters, tails and
shocks are active), and the batched patches (4096 patches, 44 M cells) on a
seeded sample of patches the oracle runs one by one.  Tolerance 1e-12 as for
the small cases (rhs_err: the change over one CFL-1 step relative to the
variable group's scale, momentum at least rho c)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2608_00746_b300 import inputs, wenoc

from gpu_util import momentum_floor, rhs_err, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _evolved_parity(case, steps):
    go = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                     bc=case.bc)
    g = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                   bc=case.bc)
    U = g.prim_to_cons(to_dev(case.V))
    g.bind(U)
    if steps:
        g.rk_step(cfl=case.cfl, nsteps=steps)
    g.sync_status()
    Uh = U.cpu().numpy()
    L = g.rhs(U).cpu().numpy()
    g.sync_status()
    del U
    torch.cuda.empty_cache()
    L_or = oracle.rhs(go, Uh)
    err = rhs_err(L, L_or, Uh, oracle.max_rate(go, Uh), case.N, case.dim,
                  momentum_floor(go, Uh))
    return err


def test_fullsize_shock_bubble_1024x512(gpu):
    err = _evolved_parity(inputs.shock_bubble_2d(nx=1024, ny=512, seed=0), 20)
    assert (err <= TOL).all(), err


def test_fullsize_circles_2048(gpu):
    err = _evolved_parity(inputs.circles_shock_2d(n=2048, seed=0), 5)
    assert (err <= TOL).all(), err


def test_fullsize_spheres_256(gpu):
    err = _evolved_parity(inputs.spheres_shock_3d(n=256, seed=0), 3)
    assert (err <= TOL).all(), err


def test_fullsize_patches_sampled(gpu):
    """All 4096 patches on the GPU, in the persistent schedule (one launch
    for the direction set) and in the window schedule (window sweeps over
    each group of equal patches); 12 seeded patches of every edge class
    checked against the oracle run on each patch as its own grid (outflow
    boundaries, cell size 1/edge)."""
    edges, states, (g3, pi, Dm) = inputs.patch_batch(npatch=4096, seed=0)
    edges = [int(e) for e in edges]
    P = wenoc.Patches(edges, g3, pi, Dm, precision="fp64")
    pooled = np.empty((P.nv, P.ncell))
    grids = {}
    for p, (e, S) in enumerate(zip(edges, states)):
        go = grids.setdefault(e, oracle.Grid((e, e, e), (1.0 / e,) * 3, g3, pi, Dm, flux="hll",
                                             bc=("outflow",) * 6))
        o = P.offsets[p]
        pooled[:, o:o + e ** 3] = oracle.prim_to_cons(go, S).reshape(P.nv, -1)
    Ud = to_dev(pooled)
    P.bind(Ud)
    L = P.rhs(Ud).cpu().numpy()
    P.sync_status()
    P.set_schedule(128, 3, 2)
    Lw = P.rhs(Ud).cpu().numpy()
    P.sync_status()
    rng = np.random.default_rng(7)
    picks = []
    for e in sorted(set(edges)):
        ids = [p for p in range(len(edges)) if edges[p] == e]
        picks += list(rng.choice(ids, 12 // len(set(edges)) + 1, replace=False))
    for p in picks:
        e = edges[p]
        go = grids[e]
        U = P.unpack(pooled, p)
        L_or = oracle.rhs(go, np.ascontiguousarray(U))
        for LL in (L, Lw):
            err = rhs_err(P.unpack(LL, p), L_or, U, oracle.max_rate(go, U), 3, 3,
                          momentum_floor(go, U))
            assert (err <= TOL).all(), (p, e, err)
