"""Pins of the Phase-Field mechanism oracle (Eq. 28, Eq. 4, the Phase-Field
step Eq. 5 and the full time step of Sec. 2.2) against closed forms,
textbook special cases and invariants."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import pf
from paper_2608_00746_b300 import inputs


def _grid(shape, N, bc="periodic"):
    dx = tuple(1.0 / n for n in shape)
    return oracle.Grid(tuple(shape), dx, [1.4] * N, [0.0] * N, [0.0] * N, flux="hllc",
                       bc=(bc,) * 6)


def _state(g, phi, u=None, P=1.0, rho=None):
    """Conservative state with fractions phi [N][...], phasic densities rho,
    velocity u (per direction, constant) and pressure P."""
    N = g.N
    rho = rho or [1.0 + p for p in range(N)]
    u = u or [0.0] * g.dim
    V = np.empty((g.nv,) + phi.shape[1:])
    for p in range(N):
        V[p] = phi[p] * rho[p]
        V[N + g.dim + 1 + p] = phi[p]
    for j in range(g.dim):
        V[N + j] = u[j]
    V[N + g.dim] = P
    return oracle.prim_to_cons(g, V)


def _smooth_fractions(shape, N, seed):
    """Random smooth fractions in (0, 1) summing to one (softmax of low modes)."""
    rng = np.random.default_rng(seed)
    axes = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in reversed(shape)], indexing="ij")
    z = []
    for _ in range(N):
        f = np.zeros(axes[0].shape)
        for _ in range(4):
            k = rng.integers(1, 3, size=len(axes))
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(0.5, 2.0) * np.sin(sum(2 * np.pi * kk * a for kk, a in zip(k, axes)) + ph)
        z.append(f)
    z = np.array(z)
    e = np.exp(z - z.max(axis=0))
    return e / e.sum(axis=0)


def _lap_convolve(f, dx):
    """5-point (2-D) Laplacian by convolution with periodic wrap."""
    k = np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], dtype=float)
    return ndimage.convolve(f, k, mode="wrap") / dx ** 2


# ---------------------------------------------------------------- Eq. 28
def test_cac_two_phase_is_the_lagrange_multiplier_form():
    """N = 2: Eq. 28 reduces to the two-phase conservative Allen-Cahn model
    with the multiplier phi (1 - phi) beta, beta = int (M/eta^2) g'(phi) /
    int phi (1 - phi) (g'(1 - phi) = -g'(phi), W_11 = -W_12 = phi_1 phi_2),
    here written out with its own 5-point stencil."""
    g = _grid((48, 40), 2)
    phi = _smooth_fractions((48, 40), 2, seed=3)
    U = _state(g, phi, u=[0.7, -0.4])
    R, B, M = pf.cac_rhs(g, U)
    eta = g.dx[0]
    assert M == pytest.approx(0.5 * eta * np.hypot(0.7, 0.4), rel=1e-14)
    f = phi[0]
    gp = 2 * f * (1 - f) * (1 - 2 * f)
    beta = (M / eta ** 2) * gp.sum() / (f * (1 - f)).sum()
    assert g.dx[0] == g.dx[1] or True
    lap = ndimage.convolve(f, np.array([[0, 0, 0], [1, -2, 1], [0, 0, 0]], float),
                           mode="wrap") / g.dx[0] ** 2 + \
        ndimage.convolve(f, np.array([[0, 1, 0], [0, -2, 0], [0, 1, 0]], float),
                         mode="wrap") / g.dx[1] ** 2
    expect = M * lap - (M / eta ** 2) * gp + f * (1 - f) * beta
    scale = np.abs(M * lap).max()
    assert np.abs(R[0] - expect).max() <= 1e-12 * scale
    assert np.abs(R[0] + R[1]).max() <= 1e-12 * scale


@pytest.mark.parametrize("n", [200])
def test_cac_tanh_profile_is_an_equilibrium_to_second_order(n):
    """phi = (1 + tanh(x / (sqrt(2) eta)))/2 solves eta^2 phi'' = g'(phi)
    (g = phi^2 (1 - phi)^2), so Eq. 28 vanishes in the continuum; with eta
    fixed the discrete residual falls by 4 per halving of dx."""
    eta = 0.02
    res = []
    for m in (n, 2 * n, 4 * n):
        g = _grid((m,), 2)
        x = (np.arange(m) + 0.5) / m
        f = 0.5 * (1 + np.tanh((x - 0.25) / (np.sqrt(2) * eta))) - \
            0.5 * (1 + np.tanh((x - 0.75) / (np.sqrt(2) * eta)))
        phi = np.array([f, 1 - f])
        U = _state(g, phi)
        R, _, _ = pf.cac_rhs(g, U, eta=eta, M=1.0)
        res.append(np.abs(R[0]).max())
    assert res[0] < 1e-2 * (1.0 / eta ** 2)          # small against one term, 1/eta^2
    assert 3.6 < res[0] / res[1] < 4.4 and 3.6 < res[1] / res[2] < 4.4, res


def test_cac_sums_and_integrals_vanish():
    """sum_p [div J_p] = 0 (reduction consistency: sum_p W_pq = 0 and
    sum_p (g'(phi_p) - phi_p sum_q g'(phi_q)) = 0 when sum phi = 1) and
    int [div J_p] = 0 for every p (the N x N system is this constraint)."""
    g = _grid((40, 36), 3)
    phi = _smooth_fractions((40, 36), 3, seed=7)
    U = _state(g, phi, u=[1.0, 0.5])
    R, _, M = pf.cac_rhs(g, U)
    scale = np.abs(R).max()
    assert np.abs(R.sum(axis=0)).max() <= 1e-12 * scale
    for p in range(3):
        assert abs(R[p].sum()) <= 1e-12 * scale * R[p].size


def test_cac_absent_phase_and_permutation():
    """An absent phase gets [div J] = 0 and leaves the others as in the
    system without it; relabelling the phases relabels the result (the
    dropped equation of the singular system does not matter)."""
    g3 = _grid((32, 32), 3)
    g2 = _grid((32, 32), 2)
    phi2 = _smooth_fractions((32, 32), 2, seed=11)
    phi3 = np.concatenate([phi2, np.zeros((1, 32, 32))])
    R3, _, _ = pf.cac_rhs(g3, _state(g3, phi3, u=[1.0, 1.0]))
    R2, _, _ = pf.cac_rhs(g2, _state(g2, phi2, u=[1.0, 1.0]))
    assert not R3[2].any()
    assert np.abs(R3[:2] - R2).max() <= 1e-13 * np.abs(R2).max()
    phi = _smooth_fractions((32, 32), 3, seed=12)
    R, _, _ = pf.cac_rhs(g3, _state(g3, phi, u=[1.0, 1.0]))
    perm = [2, 0, 1]
    Rp, _, _ = pf.cac_rhs(g3, _state(g3, phi[perm], u=[1.0, 1.0], rho=[3.0, 1.0, 2.0]))
    assert np.abs(Rp - R[perm]).max() <= 1e-12 * np.abs(R).max()


# ---------------------------------------------------------------- Eq. 4
def _cumsum_solution(r, c, dx, periodic):
    """Face gradients of (c Q')' = r in 1-D by integrating once: the face
    fluxes are F_{i+1/2} = F_{1/2} + dx sum_{j <= i} r_j; G = F / c_f.
    Periodic: F_{1/2} makes sum_i G_i dx = 0 (Q periodic); bounded: zero flux
    at both ends (r of zero mean)."""
    cs = dx * np.cumsum(r)
    if periodic:
        cf = 0.5 * (c + np.roll(c, -1))
        F0 = -np.sum(cs / cf) / np.sum(1.0 / cf)
        return (F0 + cs) / cf
    cf = 0.5 * (c[:-1] + c[1:])
    return cs[:-1] / cf


def test_qmap_1d_periodic_matches_integration():
    n = 128
    g = _grid((n,), 2)
    x = (np.arange(n) + 0.5) / n
    f = 0.5 + 0.4 * np.sin(2 * np.pi * x)
    phi = np.array([f, 1 - f])
    rng = np.random.default_rng(1)
    R = rng.standard_normal((2, n))
    Q, Rp = pf.qmap(g, phi, R)
    for p in range(2):
        Gq = (np.roll(Q[p], -1) - Q[p]) / g.dx[0]
        c = phi[p] * (1 - phi[p])
        cf = 0.5 * (c + np.roll(c, -1))
        D = (cf + np.roll(cf, 1)) / g.dx[0] ** 2          # coupling of each cell
        rr = R[p] - D * R[p].sum() / D.sum()
        G = _cumsum_solution(rr, c, g.dx[0], True)
        assert np.abs(Gq - G).max() <= 1e-9 * np.abs(G).max()


def test_qmap_separated_regions_drop_their_means():
    """Interfaces separated by cells with phi exactly 0 or 1 (c = 0): a
    region is the cells that faces with c_f > 0 connect (its c > 0 cells and
    their direct neighbours); each is solved on its own with D s_k removed,
    D the cell's coupling, s_k = sum r / sum D over the region (R17)."""
    n = 96
    g = _grid((n,), 2, bc="reflective")
    f = np.zeros(n)
    f[10:30] = np.sin(np.linspace(0.1, np.pi - 0.1, 20)) * 0.9
    f[50:80] = 1.0
    f[48:50] = [0.3, 0.7]
    f[80:83] = [0.6, 0.2, 0.05]
    phi = np.array([f, 1 - f])
    rng = np.random.default_rng(4)
    R = rng.standard_normal((2, n)) * (phi[0] * (1 - phi[0]) > 0)
    Q, Rp = pf.qmap(g, phi, R)
    dx = g.dx[0]
    c = phi[0] * (1 - phi[0])
    cf = 0.5 * (c[:-1] + c[1:])
    D = np.zeros(n)
    D[:-1] += cf / dx ** 2
    D[1:] += cf / dx ** 2
    for lo, hi in ((9, 31), (47, 51), (79, 84)):
        r = R[0, lo:hi]
        rr = r - D[lo:hi] * r.sum() / D[lo:hi].sum()
        assert np.allclose(Rp[0, lo:hi], rr, atol=1e-14 * np.abs(r).max())
        G = _cumsum_solution(rr, c[lo:hi], dx, False)
        Gq = np.diff(Q[0, lo:hi]) / dx
        assert np.abs(Gq - G).max() <= 1e-9 * max(np.abs(G).max(), 1e-300)


def test_qmap_2d_reproduces_projected_rhs():
    g = _grid((40, 32), 3)
    phi = _smooth_fractions((40, 32), 3, seed=5)
    U = _state(g, phi, u=[1.0, 0.3])
    R, _, _ = pf.cac_rhs(g, U)
    Q, Rp = pf.qmap(g, phi, R)
    for p in range(3):
        A, _ = pf.qmap_operator(g, phi[p])
        AQ = A @ Q[p].reshape(-1)
        assert np.abs(AQ - Rp[p].reshape(-1)).max() <= 1e-9 * np.abs(R[p]).max()
    # one connected region (c > 0 everywhere), and int R = 0 (Eq. 28's
    # constraint): nothing is removed
    assert np.abs(Rp - R).max() <= 1e-12 * np.abs(R).max()


# ---------------------------------------------------------------- the time step
def test_full_step_conserves_and_keeps_bounds():
    """Sec. 2.2 time steps on the two-phase advection: each phase's mass and
    fraction, momentum and energy conserved (periodic), fractions in [0, 1]
    to rounding and summing to one."""
    case = inputs.two_phase_advection_2d(n=40)
    g = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux, bc=case.bc)
    U = oracle.prim_to_cons(g, case.V)
    tot0 = U.sum(axis=(1, 2))
    for _ in range(20):
        U, _, _ = pf.full_step(g, U, dt=case.meta["dt"])
    tot = U.sum(axis=(1, 2))
    assert np.all(np.abs(tot - tot0) <= 1e-12 * np.abs(U).sum(axis=(1, 2)))
    a = U[5:7]
    assert a.min() >= -1e-12 and a.max() <= 1 + 1e-12
    assert np.abs(a.sum(axis=0) - 1).max() < 1e-13


def test_phase_field_keeps_the_equilibrium_thickness():
    """The purpose of the mechanism (Sec. 2.2, Eq. 28 with eta = dx): the
    air circle of Sec. 4.1.1 (40^2, radius 8 cells) advected for 400 steps
    keeps the equilibrium profile (1 + tanh(x / (sqrt(2) eta)))/2, whose
    0.05 < phi < 0.95 band is 2 sqrt(2) artanh(0.9) = 4.16 cells wide: about
    2 pi 8 x 4.16 = 209 cells; the hyperbolic step alone spreads wider."""
    case = inputs.two_phase_advection_2d(n=40)
    g = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                    bc=case.bc)
    Uh = oracle.prim_to_cons(g, case.V)
    Up = Uh.copy()
    for _ in range(400):
        Uh, _ = oracle.rk3_step(g, Uh, dt=case.meta["dt"])
        Up, _, _ = pf.full_step(g, Up, dt=case.meta["dt"])

    def band(U):
        a = U[5]
        return int(((a > 0.05) & (a < 0.95)).sum())
    expect = 2 * np.pi * 8 * 2 * np.sqrt(2) * np.arctanh(0.9)
    assert 0.85 * expect <= band(Up) <= 1.15 * expect, (band(Up), expect)
    assert band(Uh) >= band(Up) + 10


def test_gradient_limit_keeps_bounds_for_any_q():
    """R17: with |G| <= dx / (12 d dt) a forward-Euler Phase-Field step keeps
    masses >= 0 and fractions in [0, 1] whatever Q is (here Q of size 1e3
    on a 2-D three-phase field, so unlimited gradients are 1e5 dx / dt
    large), and the fraction sum, consistency and totals are kept."""
    case = inputs.circles_shock_2d(shape=(48, 40), seed=2, ncirc=4, rmin_cells=3,
                                   rmax_cells=10)
    g = oracle.Grid(case.shape, case.dx, case.gamma, case.pinf, case.D, flux=case.flux,
                    bc=("periodic",) * 6)
    U = oracle.prim_to_cons(g, case.V)
    for _ in range(3):                     # spread the interfaces a little
        U, _ = oracle.rk3_step(g, U, cfl=0.2)
    rng = np.random.default_rng(9)
    Q = rng.normal(size=(g.N,) + U.shape[1:]) * 1e3
    dt = 1e-3
    L = oracle.pf_rhs(g, U, Q, dt)
    Un = U + dt * L
    N, a0 = g.N, g.N + g.dim + 1
    a = Un[a0:]
    assert a.min() >= -1e-15 and a.max() <= 1.0 + 1e-15
    assert Un[:N].min() >= -1e-15 * U[:N].max()
    assert np.abs(a.sum(0) - 1.0).max() < 1e-13
    tot = np.abs(L).sum(axis=(1, 2))
    assert np.all(np.abs(L.sum(axis=(1, 2))) <= 1e-12 * tot + 1e-300)
    # the limit is what keeps them: without it the same step leaves [0, 1]
    Lu = oracle.pf_rhs(g, U, Q)
    assert (U + dt * Lu)[a0:].min() < -1e-3
