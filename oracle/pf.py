"""FP64 CPU oracle of the Phase-Field mechanism of one time step -- TEST
INFRASTRUCTURE (imported only by ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU baseline; the product path never imports it).

One time step of the paper (Sec. 2.2) is: the hyperbolic step (Eq. 3, in
``wenoc_oracle.c``) -> the volume fractions of its result as the order
parameters phi_p -> the conservative Allen-Cahn divergence [div J_p]^ of
Eq. 28 -> the auxiliary fields Q_p of Eq. 4 -> the Phase-Field step Eq. 5
(its flux in ``wenoc_oracle.c``, reading R12).  This module holds the middle
two steps and the time stepping around them, in plain numpy / scipy.sparse.

Readings (R17), where the paper is silent:
  * eta = dx of the first axis (Sec. 3.5: eta / dx = 1); M = 0.5 eta
    max_cells |u| with u the cell-average velocity of the hyperbolic result.
  * Laplacian: second-order central differences per axis (Sec. 3.5);
    boundary cells of a reflective or outflow side mirror the fraction (zero
    gradient), periodic sides wrap.  Integrals: midpoint rule (sum over
    cells times the cell volume).
  * The N x N system of Eq. 28 is singular: every column of int W sums to
    int phi_q (1 - sum phi) = 0, and W (1, ..., 1) = 0, so B is fixed up to
    a constant vector that L^c does not see.  A phase with int W_pp = 0 (absent,
    or filling the whole domain) gets B_p = 0; among the others the last one
    gets B = 0 and its equation (implied by the rest) is dropped; the
    remaining system is solved directly.
  * Eq. 4, discretised with second-order central differences: on the face
    between cells a and b the coefficient is c_f = (c_a + c_b)/2 with
    c = phi (1 - phi) for phi in [2^-52, 1 - 2^-52] and 0 otherwise (the
    degenerate coefficient; a fraction just outside [0, 1] gives 0, not a
    negative coefficient, and so do traces within one unit of rounding of
    0 or 1: the hyperbolic step leaves such traces (1e-20 .. 1e-300) in
    cells far from any interface, below the resolution of the fraction sum,
    and with them c > 0 would join those cells to the interface regions
    with coefficients of that size), and
    (A Q)_i = sum_faces c_f (Q_nbr - Q_i)/dx^2.  Reflective and outflow
    boundaries carry no flux (the mirrored cell has the same Q).
  * A is singular on every region that faces with c_f > 0 connect (its
    constants), and its right-hand side need not sum to zero there (the
    multiplier L^c moves mass between separated interfaces).  Q is the
    least-squares solution weighted by the inverse of the coupling D_i =
    sum_faces c_f/dx^2 (the diagonal of -A): on each region k the
    right-hand side minus D_i s_k, s_k = sum_k r / sum_k D, is solved
    exactly; the removed part sits where the coupling is strong, not in the
    weakly coupled edge cells.  (This is also the limit of Krylov solvers
    preconditioned by D.)  A region of one cell (D = 0) gets Q = 0.  Only
    the face gradients G = (Q_b - Q_a)/dx on faces with c_f > 0 are defined
    by this; on faces with c_f = 0 the Phase-Field flux takes G = 0 (R12,
    ``or_pf_rhs``).  The removed part is the share of [div J_p]^ that no flux
    phi_p (1 - phi_p) grad Q_p can carry.
  * Near the edges of an interface c_f is tiny and G = flux / c_f is
    unbounded (and a fraction just outside [0, 1] has c = 0 while Eq. 28
    does not vanish there).  R12's flux keeps the bounds when, summed over
    the d directions, dt |G| / dx <= 1/12 (the Gauss-Lobatto weight of
    Sec. 4.2, as for the hyperbolic step); the Phase-Field step limits each
    face gradient to |G| <= dx / (12 d dt).  The limit scales a face's
    fluxes of every variable of the phase alike (consistency and
    conservation kept); inside interfaces at the paper's time steps it is
    usually inactive.
  * The Phase-Field step (Eq. 5) is advanced with the same third-order SSP
    Runge-Kutta as the hyperbolic step (Sec. 3.5), the same time step, and
    Q held fixed over its stages (Q is computed once per time step from the
    hyperbolic result).  R13's stage rule applies.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.sparse.csgraph import connected_components

from . import Grid, cons_to_prim, pf_rhs, rk3_step

STAGE_TOL = 2.0 ** -48


def _axis(g: Grid, d: int) -> int:
    """Array axis of direction d in a [nz][ny][nx] field."""
    return g.dim - 1 - d


def _periodic(g: Grid, d: int) -> bool:
    return g.bc[2 * d] in ("periodic", 0)


def fractions(g: Grid, U: np.ndarray) -> np.ndarray:
    """phi_p = alpha_p, [N][...] (the last N conservative variables)."""
    return U[g.N + g.dim + 1:].copy()


def mobility(g: Grid, U: np.ndarray, eta: float) -> float:
    """M = 0.5 eta max |u| (Eq. 28), u = cell-average velocity."""
    V = cons_to_prim(g, U)
    u2 = sum(V[g.N + j] ** 2 for j in range(g.dim))
    return 0.5 * eta * float(np.sqrt(u2.max()))


def laplacian(g: Grid, f: np.ndarray) -> np.ndarray:
    """Second-order central Laplacian of a cell field [...] (R17 boundaries)."""
    out = np.zeros_like(f)
    for d in range(g.dim):
        ax = _axis(g, d)
        if _periodic(g, d):
            fp = np.roll(f, -1, axis=ax)
            fm = np.roll(f, 1, axis=ax)
        else:
            pad = [(0, 0)] * f.ndim
            pad[ax] = (1, 1)
            fe = np.pad(f, pad, mode="edge")
            n = f.shape[ax]
            fp = np.take(fe, np.arange(2, n + 2), axis=ax)
            fm = np.take(fe, np.arange(0, n), axis=ax)
        out += (fp - 2.0 * f + fm) / g.dx[d] ** 2
    return out


def gprime(phi: np.ndarray) -> np.ndarray:
    """g'(phi) of g(phi) = phi^2 (1 - phi)^2 (Eq. 28)."""
    return 2.0 * phi * (1.0 - phi) * (1.0 - 2.0 * phi)


def multiplier_B(Wint: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solves sum_q Wint[p, q] B_q = b_p (Eq. 28) by the R17 reading."""
    N = len(b)
    present = [p for p in range(N) if Wint[p, p] > 0.0]
    B = np.zeros(N)
    if len(present) < 2:
        return B
    keep = present[:-1]
    B[keep] = np.linalg.solve(Wint[np.ix_(keep, keep)], b[keep])
    return B


def cac_rhs(g: Grid, U: np.ndarray, eta: float = None, M: float = None):
    """[div J_p]^ of Eq. 28 for every phase, [N][...], with the order
    parameters phi_p = alpha_p of U.  eta defaults to dx (R17), M to
    0.5 eta max |u|.  Returns (R, B, M)."""
    eta = g.dx[0] if eta is None else eta
    M = mobility(g, U, eta) if M is None else M
    phi = fractions(g, U)
    N = g.N
    vol = float(np.prod(g.dx))
    gp = gprime(phi)
    S = (M / eta ** 2) * (gp - phi * gp.sum(axis=0))          # (M/eta^2)(g'(phi_p) - phi_p sum g')
    Wint = np.empty((N, N))
    for p in range(N):
        for q in range(N):
            W = phi[p] * (1.0 - phi[q]) if p == q else -phi[p] * phi[q]
            Wint[p, q] = W.sum() * vol
    b = np.array([S[p].sum() * vol for p in range(N)])
    B = multiplier_B(Wint, b)
    R = np.empty_like(phi)
    for p in range(N):
        Lc = np.zeros_like(phi[p])
        for q in range(N):
            W = phi[p] * (1.0 - phi[q]) if p == q else -phi[p] * phi[q]
            Lc += W * B[q]
        R[p] = M * laplacian(g, phi[p]) - S[p] + Lc
    return R, B, M


TRACE = 2.0 ** -52


def coefficient(phi: np.ndarray) -> np.ndarray:
    """c = phi (1 - phi) where phi is in [2^-52, 1 - 2^-52], else 0 (R17)."""
    phi = np.asarray(phi, dtype=np.float64)
    on = (phi >= TRACE) & (1.0 - phi >= TRACE)
    return np.where(on, phi * (1.0 - phi), 0.0)


def face_coefficients(g: Grid, phi: np.ndarray):
    """Per direction d: (c_f, a, b) for every face with two distinct cells,
    flat cell indices a (lower) and b (upper), c_f = (c_a + c_b)/2 with
    the coefficient of ``coefficient`` (R17)."""
    c = coefficient(phi).reshape(-1)
    idx = np.arange(phi.size).reshape(phi.shape)
    out = []
    for d in range(g.dim):
        ax = _axis(g, d)
        n = phi.shape[ax]
        if _periodic(g, d):
            a = idx
            b = np.roll(idx, -1, axis=ax)
        else:
            a = np.take(idx, np.arange(0, n - 1), axis=ax)
            b = np.take(idx, np.arange(1, n), axis=ax)
        a, b = a.reshape(-1), b.reshape(-1)
        out.append((0.5 * (c[a] + c[b]), a, b))
    return out


def qmap_operator(g: Grid, phi: np.ndarray):
    """The discrete Eq. 4 operator A (sparse, symmetric) of one phase and
    the adjacency of its faces with c_f > 0."""
    n = phi.size
    rows, cols, vals = [], [], []
    adj_r, adj_c = [], []
    for d, (cf, a, b) in enumerate(face_coefficients(g, phi)):
        w = cf / g.dx[d] ** 2
        rows += [a, b, a, b]
        cols += [b, a, a, b]
        vals += [w, w, -w, -w]
        on = w > 0.0   # the faces that carry weight in A (Eq. 4)
        adj_r += [a[on], b[on]]
        adj_c += [b[on], a[on]]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    adj = sp.csr_matrix((np.ones(sum(len(x) for x in adj_r)),
                         (np.concatenate(adj_r), np.concatenate(adj_c))), shape=(n, n))
    return A, adj


def qmap(g: Grid, phi: np.ndarray, R: np.ndarray):
    """Q_p of Eq. 4 for every phase ([N][...]), the R17 least-squares
    solution; also returns the right-hand sides after the regions' parts
    D s_k were removed (what A Q reproduces)."""
    Q = np.zeros_like(R)
    Rp = np.zeros_like(R)
    for p in range(g.N):
        A, adj = qmap_operator(g, phi[p])
        ncomp, lab = connected_components(adj, directed=False)
        Dg = -A.diagonal()
        r = R[p].reshape(-1)
        q = np.zeros_like(r)
        rp = np.zeros_like(r)
        for k in range(ncomp):
            cells = np.flatnonzero(lab == k)
            if len(cells) < 2:
                continue
            rk = r[cells] - Dg[cells] * (r[cells].sum() / Dg[cells].sum())
            rp[cells] = rk
            # the same system scaled symmetrically by D^-1/2 (unit diagonal):
            # with coefficients down to denormal sizes the unscaled
            # factorisation breaks down; the solution is unchanged
            sc = 1.0 / np.sqrt(Dg[cells])
            Ak = (sp.diags(sc) @ A[cells][:, cells] @ sp.diags(sc)).tocsc()
            rk = rk * sc
            # pin the first cell of the region (its constant is free)
            q[cells[1:]] = spla.spsolve(Ak[1:, 1:], rk[1:]) * sc[1:]
        Q[p] = q.reshape(R[p].shape)
        Rp[p] = rp.reshape(R[p].shape)
    return Q, Rp


def _stage(g: Grid, a, U0, b, U1, c, dt, L):
    """a U0 + b U1 + c dt L with R13's stage rule on masses and fractions."""
    t0, t1, t2 = a * U0, b * U1, c * dt * L
    x = t0 + t1 + t2
    tol = STAGE_TOL * (np.abs(t0) + np.abs(t1) + np.abs(t2))
    N, a0 = g.N, g.N + g.dim + 1
    for v in list(range(N)) + list(range(a0, a0 + N)):
        xv, tv = x[v], tol[v]
        xv[(xv < 0.0) & (-xv <= tv)] = 0.0
        if v >= a0:
            xv[(xv > 1.0) & (xv - 1.0 <= tv)] = 1.0
    return x


def pf_step(g: Grid, U: np.ndarray, Q: np.ndarray, dt: float) -> np.ndarray:
    """Eq. 5 over dt by SSP-RK3 with Q fixed and the face gradients limited
    for dt (R17)."""
    L = pf_rhs(g, U, Q, dt)
    U1 = _stage(g, 1.0, U, 0.0, U, 1.0, dt, L)
    L = pf_rhs(g, U1, Q, dt)
    U2 = _stage(g, 0.75, U, 0.25, U1, 0.25, dt, L)
    L = pf_rhs(g, U2, Q, dt)
    return _stage(g, 1.0 / 3.0, U, 2.0 / 3.0, U2, 2.0 / 3.0, dt, L)


def full_step(g: Grid, U: np.ndarray, cfl: float = 0.0, dt: float = 0.0, eta: float = None):
    """One time step of Sec. 2.2: hyperbolic step (Eq. 3), Eq. 28 on its
    fractions, Eq. 4, Phase-Field step (Eq. 5).  Returns (U, dt, Q)."""
    Uh, dt = rk3_step(g, U, cfl=cfl, dt=dt)
    R, _, _ = cac_rhs(g, Uh, eta=eta)
    Q, _ = qmap(g, fractions(g, Uh), R)
    return pf_step(g, Uh, Q, dt), dt, Q
