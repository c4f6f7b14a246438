"""Helpers shared by the GPU test files: build matching oracle and CUDA grids
from one seeded case, and compare fields variable by variable."""
import numpy as np

import oracle
from paper_2608_00746_b300 import inputs


def grids(case, precision="fp64", flux=None, **kw):
    import torch  # noqa: F401
    from paper_2608_00746_b300 import wenoc
    flux = flux or case.flux
    go = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=flux, bc=case.bc)
    gg = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=flux, bc=case.bc,
                    precision=precision, **kw)
    return go, gg


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel_err_per_var(A, B):
    """max |A - B| / max |B| for each variable (first axis)."""
    A = np.asarray(A).reshape(A.shape[0], -1)
    B = np.asarray(B).reshape(B.shape[0], -1)
    out = []
    for v in range(B.shape[0]):
        scale = np.abs(B[v]).max()
        d = np.abs(A[v] - B[v]).max()
        out.append(d / scale if scale > 0 else d)
    return np.array(out)


def groups(N, d):
    """Variable groups with a common scale: each phase mass, the momentum
    vector, the energy, each volume fraction."""
    g = [[p] for p in range(N)] + [list(range(N, N + d)), [N + d]]
    return g + [[N + d + 1 + p] for p in range(N)]


def momentum_floor(go, U):
    """Acoustic momentum scale max(rho c) of a state: the momentum group's
    scale when the fluid is (nearly) at rest."""
    N = go.N
    rho = np.asarray(U)[:N].sum(0)
    return float((rho * oracle.sound_speed(go, U)).max())


def state_err(A, B, N, d, mom_floor=0.0):
    """max |A - B| over a group / max |B| over that group, per variable; the
    momentum group's scale is at least mom_floor."""
    A = np.asarray(A).reshape(A.shape[0], -1)
    B = np.asarray(B).reshape(B.shape[0], -1)
    out = np.zeros(B.shape[0])
    for grp in groups(N, d):
        scale = np.abs(B[grp]).max()
        if grp[0] == N:
            scale = max(scale, mom_floor)
        for v in grp:
            d_ = np.abs(A[v] - B[v]).max()
            out[v] = d_ / scale if scale > 0 else d_
    return out


def rhs_err(L, L_or, U, rate, N, d, mom_floor=0.0):
    """dU/dt error over one CFL-1 time step (dt = 1/rate) relative to the
    group's state magnitude: max |L - L_or| dt / max |U| (momentum scale at
    least mom_floor)."""
    L = np.asarray(L).reshape(L.shape[0], -1)
    L_or = np.asarray(L_or).reshape(L_or.shape[0], -1)
    U = np.asarray(U).reshape(U.shape[0], -1)
    out = np.zeros(U.shape[0])
    for grp in groups(N, d):
        scale = np.abs(U[grp]).max()
        if grp[0] == N:
            scale = max(scale, mom_floor)
        scale *= rate
        for v in grp:
            d_ = np.abs(L[v] - L_or[v]).max()
            out[v] = d_ / scale if scale > 0 else d_
    return out


def l1_rel_per_var(A, B):
    A = np.asarray(A).reshape(A.shape[0], -1)
    B = np.asarray(B).reshape(B.shape[0], -1)
    out = []
    for v in range(B.shape[0]):
        s = np.abs(B[v]).sum()
        d = np.abs(A[v] - B[v]).sum()
        out.append(d / s if s > 0 else d)
    return np.array(out)


SMALL_CASES = {
    "slab_1d_hllc": lambda: inputs.interface_advection_1d(n=200),
    "slab_1d_absent_phase": lambda: inputs.interface_advection_1d(n=137, absent_phase=True),
    "shock_bubble_2d_ragged": lambda: inputs.shock_bubble_2d(nx=100, ny=45, seed=3),
    "five_phase_2d": lambda: inputs.multiphase_advection_2d(n=40, nphase=5),
    "spheres_3d_ragged": lambda: inputs.spheres_shock_3d(shape=(26, 19, 13), seed=1, nsph=4,
                                                        rmin_cells=2, rmax_cells=6),
    "circles_2d_n3": lambda: inputs.circles_shock_2d(shape=(70, 33), seed=2, ncirc=6,
                                                     rmin_cells=3, rmax_cells=9),
}


def l1_group(A, B, N, d):
    """sum |A - B| / sum |B| per variable group (momentum as one vector)."""
    A = np.asarray(A).reshape(A.shape[0], -1)
    B = np.asarray(B).reshape(B.shape[0], -1)
    out = np.zeros(B.shape[0])
    for grp in groups(N, d):
        s = np.abs(B[grp]).sum()
        for v in grp:
            dd = np.abs(A[v] - B[v]).sum()
            out[v] = dd / s if s > 0 else dd
    return out
