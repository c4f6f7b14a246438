"""The grid barrier of the Q-map's cooperative launch: every block passes
many barriers; when one block never arrives the others' bounded waits run
out, the call reports WC_ERR_TIMEOUT within seconds, and the context keeps
working (the next barrier run and a Q-map succeed)."""
import time

import pytest

from paper_2608_00746_b300 import inputs, wenoc

pytestmark = pytest.mark.gpu
WC_OK, WC_ERR_TIMEOUT = 0, 7


def test_barrier_passes(gpu):
    assert wenoc.grid_barrier_check(-1, rounds=2000) == WC_OK


def test_missing_block_times_out_and_context_survives(gpu):
    t0 = time.time()
    assert wenoc.grid_barrier_check(skip_block=5, rounds=10) == WC_ERR_TIMEOUT
    assert time.time() - t0 < 60.0
    assert wenoc.grid_barrier_check(-1, rounds=100) == WC_OK
    import torch
    case = inputs.two_phase_advection_2d(n=40)
    g = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                   bc=case.bc)
    U = g.prim_to_cons(torch.from_numpy(case.V).cuda())
    g.bind(U).set_pf_workspace(U.device)
    g.cac_rhs(U)
    _, iters, res = g.qmap(U, tol=1e-12)
    assert res <= 1e-12 and iters > 0


def test_bad_arguments(gpu):
    assert wenoc.lib().wc_grid_barrier_check(None, -1, 10, None) != WC_OK


def test_neighbour_barrier_passes(gpu):
    for span in (1, 3, 200):
        assert wenoc.neighbour_barrier_check(-1, span=span, rounds=1000) == WC_OK


def test_neighbour_barrier_missing_block_times_out_and_context_survives(gpu):
    """A block that leaves before the first exchange: its neighbours' bounded
    waits run out, the others stop on the error word, WC_ERR_TIMEOUT within
    seconds; then the barrier and a Q-map (which uses it) succeed."""
    t0 = time.time()
    assert wenoc.neighbour_barrier_check(skip_block=7, span=2, rounds=10) == WC_ERR_TIMEOUT
    assert time.time() - t0 < 60.0
    assert wenoc.neighbour_barrier_check(-1, span=2, rounds=100) == WC_OK
    import torch
    case = inputs.two_phase_advection_2d(n=40)
    g = wenoc.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                   bc=case.bc)
    U = g.prim_to_cons(torch.from_numpy(case.V).cuda())
    g.bind(U).set_pf_workspace(U.device)
    g.cac_rhs(U)
    _, iters, res = g.qmap(U, tol=1e-12)
    assert res <= 1e-12 and iters > 0


def test_neighbour_barrier_bad_arguments(gpu):
    L = wenoc.lib()
    assert L.wc_neighbour_barrier_check(None, 0, -1, 1, 10, None) != WC_OK
    import torch
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert L.wc_neighbour_barrier_check(wenoc._dptr(words), 4, -1, 1, 10, None) == 1
