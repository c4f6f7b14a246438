"""wc_rk_step_noalloc: SSP-RK3 stepping for callers that cannot allocate
device memory (their device memory is owned and budgeted elsewhere, or an
allocation is not allowed where they run).  Its scratch is a fixed array
inside the library; the result must match wc_rk_step with a workspace.

Collected last on purpose (file name), so a run that stops at its first
failure has already run every other test.  It also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2608_00746_b300 import inputs, wenoc

from gpu_util import grids, state_err, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(g, U, cfl=0.0, dt=0.0, nsteps=1):
    st = ctypes.c_int(-1)
    rc = wenoc.lib().wc_rk_step_noalloc(g.h, ctypes.c_void_p(U.data_ptr()), cfl, dt, nsteps,
                                        ctypes.byref(st),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, st.value


@pytest.mark.parametrize("name,precision", [("shock_bubble", "fp64"), ("shock_bubble", "mixed"),
                                            ("slab", "fp64")])
def test_noalloc_matches_workspace_path_two_calls(gpu, name, precision):
    if name == "shock_bubble":
        case = inputs.shock_bubble_2d(nx=96, ny=48, seed=7)
    else:
        case = inputs.interface_advection_1d(n=200)
    go, g_ref = grids(case, precision=precision)
    _, g_new = grids(case, precision=precision)
    U0 = oracle.prim_to_cons(go, case.V)
    U_ref = to_dev(U0)
    g_ref.bind(U_ref)
    U_new = to_dev(U0)
    cfl = case.cfl or 0.2
    for call in range(2):
        g_ref.rk_step(cfl=cfl, nsteps=3)
        rc, status = _noalloc(g_new, U_new, cfl=cfl, nsteps=3)
        assert rc == 0 and status == 0, (rc, status)
        err = state_err(U_new.cpu().numpy(), U_ref.cpu().numpy(), case.N, case.dim)
        assert (err <= 1e-12).all(), (call, err)


def test_noalloc_rejects_grids_beyond_the_scratch(gpu):
    case = inputs.shock_bubble_2d(nx=1024, ny=512, seed=0)
    _, g = grids(case)
    U = torch.zeros((g.nv, 512, 1024), dtype=torch.float64, device="cuda")
    rc, _ = _noalloc(g, U, cfl=0.2)
    assert rc == 1
    buf = ctypes.create_string_buffer(256)
    wenoc.lib().wc_last_error(g.h, buf, 256)
    assert b"too large" in buf.value
    assert not U.any()  # nothing was enqueued


@pytest.mark.parametrize("nx,ny", [(96, 48), (1024, 512)])
def test_noalloc_refuses_learned_precision_at_any_size(gpu, nx, ny):
    """The fixed scratch holds no learned-weight buffer: a learned grid is
    refused as unsupported, whether or not its stage buffers would fit."""
    case = inputs.shock_bubble_2d(nx=nx, ny=ny, seed=0)
    _, g = grids(case, precision="learned")
    U = torch.zeros((g.nv, ny, nx), dtype=torch.float64, device="cuda")
    rc, _ = _noalloc(g, U, cfl=0.2)
    assert rc == 5  # WC_ERR_UNSUPPORTED
    buf = ctypes.create_string_buffer(256)
    wenoc.lib().wc_last_error(g.h, buf, 256)
    assert b"learned" in buf.value
    assert not U.any()
