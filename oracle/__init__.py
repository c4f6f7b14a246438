"""FP64 CPU oracle of the WENO-C operator -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it; the two implementations share no code.

The arithmetic lives in ``wenoc_oracle.c`` (plain C, FP64, no fused
multiply-add); this module compiles it with gcc and wraps it with ctypes and
numpy arrays.  Every function cites the paper passage it follows in the C
source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wenoc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXP = 8
BC = {"periodic": 0, "reflective": 1, "outflow": 2}
FLUX = {"hll": 0, "hllc": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over pencils, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("N", ctypes.c_int),
        ("gamma", ctypes.c_double * MAXP),
        ("pinf", ctypes.c_double * MAXP),
        ("D", ctypes.c_double * MAXP),
        ("pmin", ctypes.c_double * MAXP),
        ("flux", ctypes.c_int),
        ("weights", ctypes.c_int),
        ("js_eps", ctypes.c_double),
        ("coupled", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("energy_limiter", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("consistent", ctypes.c_int),
        ("kmodel", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        gp = ctypes.POINTER(_Grid)
        for name, args in {
            "or_rhs": [gp, dp, dp],
            "or_rk3_step": [gp, dp, ctypes.c_double, ctypes.c_double, dp],
            "or_pf_rhs": [gp, dp, dp, ctypes.c_double, dp],
            "or_pf_flux": [gp, ctypes.c_int, dp, dp, dp, dp, dp, dp],
            "or_faces": [gp, ctypes.c_int, dp, dp, dp, dp],
            "or_limit": [gp, ctypes.c_long, dp, dp, dp, dp, dp, dp],
            "or_cons_to_prim": [gp, ctypes.c_long, dp, dp],
            "or_prim_to_cons": [gp, ctypes.c_long, dp, dp],
            "or_psi": [gp, ctypes.c_long, dp, dp],
            "or_sound_speed": [gp, ctypes.c_long, dp, dp],
            "or_max_rate": [gp, dp, dp],
            "or_flux": [gp, ctypes.c_int, dp, dp, dp, dp, dp, dp],
            "or_weno5_parts": [dp, dp, dp],
            "or_wenow_weights": [dp, dp],
            "or_wenojs_weights": [dp, ctypes.c_double, dp],
            "or_nv": [gp],
            "or_num_threads": [],
        }.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        for name, args in {
            "or_set_num_threads": [ctypes.c_int],
            "or_r13_set_stage_tol": [ctypes.c_double],
            "or_r13_reset": [],
            "or_r13_stats": [dp],
            "or_rk_stage": [gp, ctypes.c_double, dp, ctypes.c_double, dp, ctypes.c_double,
                            ctypes.c_double, dp, dp],
        }.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = None
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} returned status {rc}")


@dataclass
class Grid:
    """Uniform grid + materials.  ``shape`` is (nx,), (nx, ny) or (nx, ny, nz)."""
    shape: tuple
    dx: tuple
    gamma: list
    pinf: list
    D: list = None
    pmin: list = None
    flux: str = "hll"
    bc: tuple = ("periodic",) * 6
    weights: str = "w"          # "w" (Eq. 15) or "js" (comparator)
    js_eps: float = 1e-6
    coupled: bool = True        # Eq. 16
    limiter: bool = True        # Eq. 17-20
    energy_limiter: bool = True  # Eq. 21
    scheme: str = "c"           # "c": Eq. 19 (WENO-C); "cl": Eq. 23-25 (WENO-CL)
    kmodel: str = "allaire"     # K_p of Eq. 2-3: "allaire" (0) or "kapila" (R15)
    _c: _Grid = field(default=None, repr=False)

    def __post_init__(self):
        N = len(self.gamma)
        if self.D is None:
            self.D = [0.0] * N
        if self.pmin is None:
            self.pmin = default_pmin(self.pinf)
        g = _Grid()
        g.dim = len(self.shape)
        for a in range(3):
            g.n[a] = self.shape[a] if a < g.dim else 1
            g.dx[a] = self.dx[a] if a < g.dim else 1.0
        g.N = N
        for p in range(N):
            g.gamma[p] = self.gamma[p]
            g.pinf[p] = self.pinf[p]
            g.D[p] = self.D[p]
            g.pmin[p] = self.pmin[p]
        g.flux = FLUX[self.flux]
        g.weights = 0 if self.weights == "w" else 1
        g.js_eps = self.js_eps
        g.coupled = int(self.coupled)
        g.limiter = int(self.limiter)
        g.energy_limiter = int(self.energy_limiter)
        for k in range(6):
            g.bc[k] = BC[self.bc[k]] if isinstance(self.bc[k], str) else int(self.bc[k])
        g.consistent = {"c": 0, "cl": 1}[self.scheme]
        g.kmodel = {"allaire": 0, "kapila": 1}[self.kmodel]
        self._c = g

    @property
    def N(self):
        return len(self.gamma)

    @property
    def dim(self):
        return len(self.shape)

    @property
    def nv(self):
        return 2 * self.N + self.dim + 1

    @property
    def ncell(self):
        return int(np.prod(self.shape))

    def state_shape(self):
        # [NV][nz][ny][nx]: x fastest
        return (self.nv,) + tuple(reversed(self.shape))

    def ref(self):
        return ctypes.byref(self._c)


def default_pmin(pinf):
    """Minimum pressures of Eq. 9 when the caller gives none: -(1 - 1e-3) Pinf_p
    for stiffened phases and 0 for ideal gases (the paper leaves them to the
    user, Sec. 2.2.2)."""
    return [-(1.0 - 1e-3) * pi if pi > 0 else 0.0 for pi in pinf]


def rhs(g: Grid, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    L = np.empty_like(U)
    _check(lib().or_rhs(g.ref(), _p(U), _p(L)), "or_rhs")
    return L


def pf_rhs(g: Grid, U: np.ndarray, Q: np.ndarray, dt_limit: float = 0.0) -> np.ndarray:
    """dU/dt of the Phase-Field step (Eq. 5) for the auxiliary fields Q [N][...];
    dt_limit > 0 limits the face gradients for that time step (R17)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    L = np.empty_like(U)
    _check(lib().or_pf_rhs(g.ref(), _p(U), _p(Q), float(dt_limit), _p(L)), "or_pf_rhs")
    return L


def pf_flux(g: Grid, direction, UL, VL, UR, VR, G):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (UL, VL, UR, VR, G)]
    F = np.empty(g.nv)
    lib().or_pf_flux(g.ref(), direction, *[_p(a) for a in arrs], _p(F))
    return F


def rk3_step(g: Grid, U: np.ndarray, cfl: float = 0.5, dt: float = 0.0):
    """One SSP-RK3 step; returns (U_new, dt_used)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    out = ctypes.c_double(0.0)
    _check(lib().or_rk3_step(g.ref(), _p(U), cfl, dt, ctypes.byref(out)), "or_rk3_step")
    return U, out.value


def faces(g: Grid, U: np.ndarray, direction: int):
    U = np.ascontiguousarray(U, dtype=np.float64)
    UL = np.empty_like(U)
    UR = np.empty_like(U)
    TH = np.empty((3,) + U.shape[1:], dtype=np.float64)
    _check(lib().or_faces(g.ref(), direction, _p(U), _p(UL), _p(UR), _p(TH)), "or_faces")
    return UL, UR, TH


def limit(g: Grid, Ubar, VL, VR):
    """Eq. 17-21 on raw primitive face values of independent cells ([NV][n])."""
    Ubar, VL, VR = (np.ascontiguousarray(a, dtype=np.float64) for a in (Ubar, VL, VR))
    n = Ubar.shape[1]
    UL = np.empty_like(Ubar)
    UR = np.empty_like(Ubar)
    TH = np.empty((3, n))
    _check(lib().or_limit(g.ref(), n, _p(Ubar), _p(VL), _p(VR), _p(UL), _p(UR), _p(TH)),
           "or_limit")
    return UL, UR, TH


def _cellwise(fname, g, A, nout=None):
    A = np.ascontiguousarray(A, dtype=np.float64)
    flat = A.reshape(A.shape[0], -1)
    n = flat.shape[1]
    out = np.empty((nout, n) if nout else flat.shape)
    _check(getattr(lib(), fname)(g.ref(), n, _p(flat), _p(out)), fname)
    return out


def cons_to_prim(g, U):
    return _cellwise("or_cons_to_prim", g, U).reshape(np.shape(U))


def prim_to_cons(g, V):
    return _cellwise("or_prim_to_cons", g, V).reshape(np.shape(V))


def psi(g, U):
    return _cellwise("or_psi", g, U, 1)[0].reshape(np.shape(U)[1:])


def sound_speed(g, U):
    return _cellwise("or_sound_speed", g, U, 1)[0].reshape(np.shape(U)[1:])


def max_rate(g, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = ctypes.c_double(0.0)
    _check(lib().or_max_rate(g.ref(), _p(U), ctypes.byref(out)), "or_max_rate")
    return out.value


def heat_capacities(g: Grid, rho, P0, T0):
    """C_p^T of the thermal-equilibrium rule of Sec. 4.1.1: C_p^T = (A_p P0 +
    B_p - B_p^T) / (rho_p T0), with A_p = 1/(gamma_p - 1), B_p = gamma_p
    Pinf_p/(gamma_p - 1) and B_p^T = Pinf_p (Eq. 26), so a state at uniform
    P0 with phasic densities rho_p has T = T0 in every phase."""
    out = []
    for p in range(g.N):
        A = 1.0 / (g.gamma[p] - 1.0)
        B = g.gamma[p] * g.pinf[p] / (g.gamma[p] - 1.0)
        out.append((A * P0 + B - g.pinf[p]) / (rho[p] * T0))
    return out


def temperature(g: Grid, U, cT):
    """Mixture temperature of Eq. 29 (numpy, per cell): (rho E - |rho u|^2 /
    (2 rho) - sum_p B_p^T alpha_p - sum_p D_p (alpha rho)_p) / sum_p C_p^T
    (alpha rho)_p, B_p^T = Pinf_p (Eq. 26)."""
    N, d = g.N, g.dim
    rho = sum(U[p] for p in range(N))
    mom2 = sum(U[N + j] ** 2 for j in range(d))
    num = U[N + d] - 0.5 * mom2 / rho
    den = np.zeros_like(rho)
    for p in range(N):
        num = num - g.pinf[p] * U[N + d + 1 + p] - g.D[p] * U[p]
        den = den + cT[p] * U[p]
    return num / den


def flux(g: Grid, direction, UL, VL, UR, VR):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (UL, VL, UR, VR)]
    F = np.empty(g.nv)
    uh = ctypes.c_double(0.0)
    _check(lib().or_flux(g.ref(), direction, *[_p(a) for a in arrs], _p(F), ctypes.byref(uh)),
           "or_flux")
    return F, uh.value


def weno5_parts(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    q = np.empty(3)
    b = np.empty(3)
    lib().or_weno5_parts(_p(f), _p(q), _p(b))
    return q, b


def wenow_weights(beta):
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    w = np.empty(3)
    lib().or_wenow_weights(_p(beta), _p(w))
    return w


def wenojs_weights(beta, eps):
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    w = np.empty(3)
    lib().or_wenojs_weights(_p(beta), eps, _p(w))
    return w


def set_num_threads(n):
    """Threads of the oracle's parallel sweeps (OpenMP)."""
    lib().or_set_num_threads(int(n))


def num_threads():
    return lib().or_num_threads()


# ---------------------------------------------------------------- R13 hooks
def r13_reset():
    """Clears R13's bookkeeping (face residues and the stage histogram)."""
    lib().or_r13_reset()


def r13_stats():
    """R13's bookkeeping since the last reset: ``face_n`` face values the
    face rule set to 0, ``face_max`` their largest |x| / fbar, and ``hist``
    {log2 bin: count} of the stage values found outside a bound, binned by
    floor(log2(excursion / sum of the stage terms' magnitudes))."""
    out = np.zeros(68)
    lib().or_r13_stats(_p(out))
    hist = {b - 64: int(out[2 + b]) for b in range(66) if out[2 + b] > 0}
    return {"face_n": int(out[0]), "face_max": float(out[1]), "hist": hist}


def set_stage_tol(tol):
    """Tolerance of R13's stage rule (relative to the sum of the terms'
    magnitudes); 2^-48 is the oracle's.  For tests that run the method with
    another one."""
    lib().or_r13_set_stage_tol(float(tol))


def rk_stage(g: Grid, a, U0, b, U1, c, dt, L):
    """One stage a U0 + b U1 + c dt L with R13's stage rule (the bounded
    variables are the masses and fractions)."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    U1 = np.ascontiguousarray(U1, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    out = np.empty_like(U0)
    lib().or_rk_stage(g.ref(), float(a), _p(U0), float(b), _p(U1), float(c), float(dt), _p(L),
                      _p(out))
    return out
