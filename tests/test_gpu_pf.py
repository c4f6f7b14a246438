"""Phase-Field step operator (Eq. 5) on the GPU vs the oracle."""
import numpy as np
import pytest

import oracle

from gpu_util import SMALL_CASES, grids, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt_limit", [0.0, 2e-3])
@pytest.mark.parametrize("name", sorted(SMALL_CASES))
def test_pf_rhs_parity(gpu, name, dt_limit):
    """Random Q (so many face gradients are large): decoupled faces (both
    cells at phi = 0 or 1) take G = 0, and with dt_limit the gradients are
    limited to dx / (12 d dt_limit)."""
    case = SMALL_CASES[name]()
    go, gg = grids(case)
    U = oracle.prim_to_cons(go, case.V)
    rng = np.random.default_rng(11)
    Q = rng.normal(size=(case.N,) + U.shape[1:]) * 0.05
    L_or = oracle.pf_rhs(go, U, Q, dt_limit)
    Ud = to_dev(U)
    gg.bind(Ud)
    L = gg.rhs_pf(Ud, to_dev(Q), dt_limit=dt_limit).cpu().numpy()
    gg.sync_status()
    A = L.reshape(L.shape[0], -1)
    B = L_or.reshape(L.shape[0], -1)
    scale = np.abs(B).max(1)
    # momentum components share one scale
    N, d = case.N, case.dim
    scale[N:N + d] = scale[N:N + d].max()
    err = np.abs(A - B).max(1) / np.maximum(scale, 1e-300)
    assert (err <= 1e-12).all(), err


def test_pf_constant_q_gives_zero(gpu):
    case = SMALL_CASES["circles_2d_n3"]()
    go, gg = grids(case)
    U = to_dev(oracle.prim_to_cons(go, case.V))
    gg.bind(U)
    Q = to_dev(np.full((case.N,) + tuple(U.shape[1:]), 2.5))
    assert not gg.rhs_pf(U, Q).any()
