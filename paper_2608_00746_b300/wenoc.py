"""Thin Python binding of the C ABI in ``include/wenoc.h``.

Argument marshalling only: every step of the operator runs in the CUDA
library ``libwenoc.so`` built in-tree for sm_103a.  PyTorch supplies device
memory (the caller's state and workspace tensors) and the CUDA stream.  There
is no CPU fallback: importing this module without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwenoc.so")

MAX_PHASE = 8
BC = {"periodic": 0, "reflective": 1, "outflow": 2}
FLUX = {"hll": 0, "hllc": 1}
PREC = {"fp64": 0, "mixed": 1, "learned": 2}
SCHEME = {"c": 0, "cl": 1, "w": 2, "js": 3}
KMODEL = {"allaire": 0, "kapila": 1}
STATUS = {0: "WC_OK", 1: "WC_ERR_ARG", 2: "WC_ERR_CUDA", 3: "WC_ERR_INADMISSIBLE",
          4: "WC_ERR_NAN", 5: "WC_ERR_UNSUPPORTED", 6: "WC_ERR_STATE", 7: "WC_ERR_TIMEOUT"}


class WcError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("nphase", ctypes.c_int),
        ("gamma", ctypes.c_double * MAX_PHASE),
        ("pinf", ctypes.c_double * MAX_PHASE),
        ("D", ctypes.c_double * MAX_PHASE),
        ("pmin", ctypes.c_double * MAX_PHASE),
        ("flux", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("energy_limiter", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("seg", ctypes.c_int),
        ("block", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("kmodel", ctypes.c_int),
        ("js_eps", ctypes.c_double),
    ]


class PatchesDesc(ctypes.Structure):
    _fields_ = [
        ("nphase", ctypes.c_int),
        ("gamma", ctypes.c_double * MAX_PHASE),
        ("pinf", ctypes.c_double * MAX_PHASE),
        ("D", ctypes.c_double * MAX_PHASE),
        ("pmin", ctypes.c_double * MAX_PHASE),
        ("flux", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("energy_limiter", ctypes.c_int),
        ("npatch", ctypes.c_int),
        ("kmodel", ctypes.c_int),
    ]


# name -> (restype, argtypes)
_VP = ctypes.c_void_p
_SIGS = {
    "wc_temperature": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double), _VP, _VP]),
    "wc_pf_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "wc_set_pf_workspace": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "wc_cac_rhs": (ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.c_double, _VP, _VP]),
    "wc_qmap": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _VP]),
    "wc_pf_step": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP]),
    "wc_step": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP]),
    "wc_pf_band": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int)]),
    "wc_pf_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_double)]),
    "wc_pf_q": (_VP, [_VP]),
    "wc_init_grid": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.POINTER(_VP)]),
    "wc_destroy": (None, [_VP]),
    "wc_nvar": (ctypes.c_int, [_VP]),
    "wc_ncell": (ctypes.c_long, [_VP]),
    "wc_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "wc_face_buffer_bytes": (ctypes.c_size_t, [_VP]),
    "wc_prim_buffer_bytes": (ctypes.c_size_t, [_VP]),
    "wc_patches_prim_buffer_bytes": (ctypes.c_size_t, [_VP]),
    "wc_set_state": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_size_t]),
    "wc_check_state": (ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.POINTER(ctypes.c_long),
                                      ctypes.POINTER(ctypes.c_long), _VP]),
    "wc_upload_state": (ctypes.c_int, [_VP, _VP, _VP]),
    "wc_rk_step_host": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _VP]),
    "wc_download_state": (ctypes.c_int, [_VP, _VP, _VP]),
    "wc_prim_to_cons": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "wc_cons_to_prim": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "wc_rhs": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "wc_faces": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "wc_compute_dt": (ctypes.c_int, [_VP, ctypes.c_double, _VP, _VP]),
    "wc_rhs_pf": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _VP, _VP]),
    "wc_rk_step": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_double), _VP]),
    "wc_limit": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_long, _VP, _VP, _VP, _VP, _VP, _VP,
                                _VP]),
    "wc_sync_status": (ctypes.c_int, [_VP, _VP]),
    "wc_last_error": (None, [_VP, ctypes.c_char_p, ctypes.c_size_t]),
    "wc_fp64_peak_kernel": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP,
                                           ctypes.POINTER(ctypes.c_double), _VP]),
    "wc_convert_f32": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_long, _VP]),
    "wc_grid_barrier_check": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP]),
    "wc_neighbour_barrier_words": (ctypes.c_size_t, []),
    "wc_neighbour_barrier_check": (ctypes.c_int, [_VP, ctypes.c_size_t, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, _VP]),
    "wc_sweep_timing_begin": (ctypes.c_int, [_VP, ctypes.c_int]),
    "wc_sweep_timing_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
    "wc_patches_init": (ctypes.c_int, [ctypes.POINTER(PatchesDesc), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(_VP)]),
    "wc_patches_destroy": (None, [_VP]),
    "wc_patches_ncell": (ctypes.c_long, [_VP]),
    "wc_patches_offset": (ctypes.c_long, [_VP, ctypes.c_int]),
    "wc_patches_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "wc_patches_face_buffer_bytes": (ctypes.c_size_t, [_VP]),
    "wc_patches_set_state": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "wc_patches_set_schedule": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "wc_patches_rk_step": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, _VP]),
    "wc_patches_rhs": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "wc_patches_prim_to_cons": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "wc_patches_sync_status": (ctypes.c_int, [_VP, _VP]),
    "wc_patches_autotune": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, _VP,
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]),
    "wc_patches_last_error": (None, [_VP, ctypes.c_char_p, ctypes.c_size_t]),
    "wc_rk_step_noalloc": (ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int), _VP]),
    "wc_mlp_param_bytes": (ctypes.c_size_t, []),
    "wc_mlp_nparam": (ctypes.c_int, []),
    "wc_mlp_init_master": (ctypes.c_int, [_VP, ctypes.c_ulonglong]),
    "wc_mlp_pack": (ctypes.c_int, [_VP, _VP, _VP]),
    "wc_mlp_features": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_long, _VP, _VP, _VP, _VP,
                                       ctypes.c_long, _VP]),
    "wc_mlp_forward": (ctypes.c_int, [_VP, ctypes.c_long, _VP, _VP, _VP, _VP]),
    "wc_mlp_infer": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "wc_mlp_gradients": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "wc_mlp_adam": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_float, ctypes.c_int, _VP]),
    "wc_mlp_train_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP,
                                         ctypes.c_float, ctypes.c_int, _VP, _VP, _VP]),
    "wc_set_mlp": (ctypes.c_int, [_VP, _VP, ctypes.c_float, _VP]),
}

_lib = None


def lib():
    """Loads ``libwenoc.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run python -m paper_2608_00746_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dptr(t):
    """Device pointer of any contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_pmin(pinf):
    """Minimum phasic pressures of Eq. 9 when none are given: -(1 - 1e-3) Pinf_p
    for stiffened phases, 0 for ideal gases."""
    return [-(1.0 - 1e-3) * p if p > 0 else 0.0 for p in pinf]


class Grid:
    """Handle of one uniform grid with its materials and scheme options."""

    def __init__(self, shape, dx, gamma, pinf, D=None, pmin=None, flux="hll",
                 bc=("periodic",) * 6, precision="fp64", energy_limiter=True, seg=0, block=0,
                 blocks_per_sm=0, scheme="c", kmodel="allaire", js_eps=1e-6):
        N = len(gamma)
        d = GridDesc()
        d.dim = len(shape)
        for a in range(3):
            d.n[a] = int(shape[a]) if a < d.dim else 1
            d.dx[a] = float(dx[a]) if a < d.dim else 1.0
        d.nphase = N
        D = list(D) if D is not None else [0.0] * N
        pmin = list(pmin) if pmin is not None else default_pmin(pinf)
        for p in range(N):
            d.gamma[p], d.pinf[p], d.D[p], d.pmin[p] = gamma[p], pinf[p], D[p], pmin[p]
        d.flux = FLUX[flux]
        d.precision = PREC[precision]
        d.energy_limiter = int(bool(energy_limiter))
        for k in range(6):
            d.bc[k] = BC[bc[k]] if isinstance(bc[k], str) else int(bc[k])
        d.seg = int(seg)
        d.block = int(block)
        d.blocks_per_sm = int(blocks_per_sm)
        d.scheme = SCHEME[scheme]
        d.kmodel = KMODEL[kmodel]
        d.js_eps = float(js_eps)
        self.desc = d
        self.shape = tuple(shape)
        h = _VP()
        self._check(lib().wc_init_grid(ctypes.byref(d), ctypes.byref(h)), None)
        self.h = h
        self.nv = lib().wc_nvar(h)
        self.ncell = lib().wc_ncell(h)
        self.U = None
        self.ws = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.wc_destroy(h)
            self.h = None

    def _check(self, st, h="self"):
        if st != 0:
            msg = ""
            if h is not None and getattr(self, "h", None) is not None:
                buf = ctypes.create_string_buffer(256)
                lib().wc_last_error(self.h, buf, 256)
                msg = buf.value.decode()
            raise WcError(st, msg)

    @property
    def state_shape(self):
        return (self.nv,) + tuple(reversed(self.shape))

    @property
    def N(self):
        return self.desc.nphase

    def workspace_bytes(self):
        return lib().wc_workspace_bytes(self.h)

    def new_workspace(self, device="cuda", faces=True, prim=True):
        """A workspace tensor; faces=False leaves out the split sweep's face
        buffer (the single-pass sweep runs then), and with it prim=False the
        primitive slots (each sweep converts its cells then)."""
        nb = self.workspace_bytes()
        if not faces:
            nb -= lib().wc_face_buffer_bytes(self.h)
            if not prim:
                nb -= lib().wc_prim_buffer_bytes(self.h)
        return torch.empty((nb + 7) // 8, dtype=torch.float64, device=device)

    def bind(self, U, workspace=None, validate=False, sum_tol=1e-10):
        """Binds the device state tensor (advanced in place by rk_step);
        validate: check it against the admissible set of Eq. 8 first
        (WcError WC_ERR_INADMISSIBLE when a cell is outside)."""
        if workspace is None:
            workspace = self.new_workspace(U.device)
        self.U, self.ws = U, workspace
        self._check(lib().wc_set_state(self.h, _ptr(U), _ptr(workspace),
                                       workspace.numel() * 8))
        if validate:
            self.check_state(U, sum_tol)
        return self

    def check_state(self, U, sum_tol=1e-10, stream=None):
        """(cells outside the admissible set, first such cell); raises
        WcError WC_ERR_INADMISSIBLE when there are any."""
        nb, first = ctypes.c_long(0), ctypes.c_long(0)
        st = lib().wc_check_state(self.h, _ptr(U), float(sum_tol), ctypes.byref(nb),
                                  ctypes.byref(first), _stream(stream))
        self._check(st)
        return nb.value, first.value

    def prim_to_cons(self, V, U=None, stream=None):
        U = torch.empty_like(V) if U is None else U
        self._check(lib().wc_prim_to_cons(self.h, _ptr(V), _ptr(U), _stream(stream)))
        return U

    def cons_to_prim(self, U, V=None, stream=None):
        V = torch.empty_like(U) if V is None else V
        self._check(lib().wc_cons_to_prim(self.h, _ptr(U), _ptr(V), _stream(stream)))
        return V

    def rhs(self, U, L=None, stream=None):
        L = torch.empty_like(U) if L is None else L
        self._check(lib().wc_rhs(self.h, _ptr(U), _ptr(L), _stream(stream)))
        return L

    def faces(self, U, direction, stream=None):
        """The limited conservative face states (U^L_{i+1/2}, U^R_{i-1/2}) of
        one direction's sweep, each shaped like U."""
        UL = torch.empty_like(U)
        UR = torch.empty_like(U)
        self._check(lib().wc_faces(self.h, int(direction), _ptr(U), _ptr(UL), _ptr(UR),
                                   _stream(stream)))
        return UL, UR

    def rhs_pf(self, U, Q, L=None, dt_limit=0.0, stream=None):
        """Phase-Field step operator (Eq. 5) for auxiliary fields Q [N][...];
        dt_limit > 0 limits the face gradients for that time step."""
        L = torch.empty_like(U) if L is None else L
        self._check(lib().wc_rhs_pf(self.h, _ptr(U), _ptr(Q), float(dt_limit), _ptr(L),
                                    _stream(stream)))
        return L

    def compute_dt(self, cfl, out=None, stream=None):
        out = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
        self._check(lib().wc_compute_dt(self.h, cfl, _ptr(out), _stream(stream)))
        return out

    def rk_step(self, cfl=0.0, dt=0.0, nsteps=1, want_dt=False, stream=None):
        dth = ctypes.c_double(0.0)
        self._check(lib().wc_rk_step(self.h, float(cfl), float(dt), int(nsteps),
                                     ctypes.byref(dth) if want_dt else None, _stream(stream)))
        return dth.value if want_dt else None

    def rk_step_host(self, U_in, U_out=None, cfl=0.0, dt=0.0, nsteps=1, stream=None):
        """Upload U_in (host, [NV][ncell], pinned for overlap), nsteps SSP-RK3
        steps, download into U_out (default U_in); asynchronous on stream."""
        U_out = U_in if U_out is None else U_out
        for t in (U_in, U_out):
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous() \
                    or t.numel() != self.nv * self.ncell:
                raise ValueError("host buffers: contiguous CPU float64 of NV x ncell values")
        self._check(lib().wc_rk_step_host(self.h, ctypes.c_void_p(U_in.data_ptr()),
                                          ctypes.c_void_p(U_out.data_ptr()), float(cfl), float(dt),
                                          int(nsteps), _stream(stream)))
        return U_out

    def upload(self, U_host, stream=None):
        self._check(lib().wc_upload_state(self.h, ctypes.c_void_p(U_host.data_ptr()),
                                          _stream(stream)))

    def download(self, U_host, stream=None):
        self._check(lib().wc_download_state(self.h, ctypes.c_void_p(U_host.data_ptr()),
                                            _stream(stream)))

    def limit(self, direction, Ubar, VL, VR, stream=None, want_theta=True):
        n = Ubar.shape[1]
        UL = torch.empty_like(Ubar)
        UR = torch.empty_like(Ubar)
        TH = torch.empty((3, n), dtype=torch.float64, device=Ubar.device) if want_theta else None
        self._check(lib().wc_limit(self.h, direction, n, _ptr(Ubar), _ptr(VL), _ptr(VR),
                                   _ptr(UL), _ptr(UR), _ptr(TH), _stream(stream)))
        return UL, UR, TH

    def sweep_timing_begin(self, max_launches):
        self._check(lib().wc_sweep_timing_begin(self.h, int(max_launches)))

    def sweep_timing_read(self):
        n = ctypes.c_int(0)
        tot = ctypes.c_double(0.0)
        mx = ctypes.c_double(0.0)
        self._check(lib().wc_sweep_timing_read(self.h, ctypes.byref(n), ctypes.byref(tot),
                                               ctypes.byref(mx)))
        return n.value, tot.value, mx.value

    def sync_status(self, stream=None):
        self._check(lib().wc_sync_status(self.h, _stream(stream)))

    def temperature(self, U, cT, T=None, stream=None):
        """Mixture temperature of Eq. 29 per cell for heat capacities cT[N]."""
        T = torch.empty(tuple(U.shape[1:]), dtype=torch.float64, device=U.device) \
            if T is None else T
        arr = (ctypes.c_double * self.N)(*[float(c) for c in cT])
        self._check(lib().wc_temperature(self.h, _ptr(U), arr, _ptr(T), _stream(stream)))
        return T

    # Phase-Field mechanism (Eq. 28, Eq. 4, Eq. 5) ---------------------------
    def set_pf_workspace(self, device="cuda"):
        """Allocates and binds the mechanism's scratch (torch memory)."""
        n = (lib().wc_pf_workspace_bytes(self.h) + 7) // 8
        self.pfws = torch.empty(n, dtype=torch.float64, device=device)
        self._check(lib().wc_set_pf_workspace(self.h, _ptr(self.pfws), n * 8))
        return self

    def cac_rhs(self, U, eta=0.0, M=-1.0, R=None, stream=None):
        """[div J_p]^ of Eq. 28, [N][...] (eta <= 0: dx; M < 0: 0.5 eta max|u|)."""
        R = torch.empty((self.N,) + tuple(U.shape[1:]), dtype=torch.float64,
                        device=U.device) if R is None else R
        self._check(lib().wc_cac_rhs(self.h, _ptr(U), float(eta), float(M), _ptr(R),
                                     _stream(stream)))
        return R

    def qmap(self, U, R=None, Q=None, tol=1e-12, maxit=20000, warm=False, stream=None):
        """Q of Eq. 4 ([N][...]) for the fractions of U and right-hand sides R
        (None: the last cac_rhs); warm: start from the Q given; returns (Q,
        CG iterations, residual)."""
        if Q is None:
            warm = False
            Q = torch.empty((self.N,) + tuple(U.shape[1:]), dtype=torch.float64, device=U.device)
        it, res = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(lib().wc_qmap(self.h, _ptr(U), _dptr(R), _ptr(Q), float(tol), int(maxit),
                                  int(bool(warm)), ctypes.byref(it), ctypes.byref(res),
                                  _stream(stream)))
        return Q, it.value, res.value

    def pf_step(self, Q, dt, stream=None):
        """The Phase-Field step (Eq. 5) over dt on the bound state."""
        self._check(lib().wc_pf_step(self.h, _ptr(Q), float(dt), _stream(stream)))

    def step(self, cfl=0.0, dt=0.0, nsteps=1, tol=1e-12, maxit=20000, want_dt=False,
             stream=None):
        """nsteps full time steps (hyperbolic step, Eq. 28, Eq. 4, Phase-Field step)."""
        dth = ctypes.c_double(0.0)
        self._check(lib().wc_step(self.h, float(cfl), float(dt), int(nsteps), float(tol),
                                  int(maxit), ctypes.byref(dth) if want_dt else None,
                                  _stream(stream)))
        return dth.value if want_dt else None

    def pf_stats(self):
        it, lr, res = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(lib().wc_pf_stats(self.h, ctypes.byref(it), ctypes.byref(lr),
                                      ctypes.byref(res)))
        return it.value, lr.value, res.value

    def pf_band(self):
        """(unknowns per phase, unknowns a thread kept in registers) of the
        last Q-map."""
        arr = (ctypes.c_int * 8)()
        pt = ctypes.c_int(0)
        self._check(lib().wc_pf_band(self.h, arr, ctypes.byref(pt)))
        return [arr[p] for p in range(self.N)], pt.value

    # learned weights ------------------------------------------------------
    def set_mlp(self, params, tau=1e-4, counters=None):
        """Binds the surrogate's parameter block (uint8 CUDA tensor) for a
        grid of precision "learned"; counters: optional int64 CUDA tensor [2]
        accumulating (face sides decided, fallbacks to the plain weights)."""
        self._mlp_keep = (params, counters)
        self._check(lib().wc_set_mlp(self.h, _dptr(params), float(tau), _dptr(counters)))

    def mlp_features(self, U, direction, X, T=None, row0=0, lst=None, count=None, stream=None):
        cap = 0 if lst is None else lst.numel()
        self._check(lib().wc_mlp_features(self.h, _ptr(U), int(direction), int(row0), _dptr(X),
                                          _dptr(T), _dptr(lst), _dptr(count), cap,
                                          _stream(stream)))

    def mlp_infer(self, U, direction, params, W=None, status=None, stream=None):
        W = torch.empty((18, self.ncell), dtype=torch.float32, device=U.device) if W is None \
            else W
        status = torch.zeros(1, dtype=torch.int32, device=U.device) if status is None else status
        self._check(lib().wc_mlp_infer(self.h, _ptr(U), int(direction), _dptr(params), _dptr(W),
                                       _dptr(status), _stream(stream)))
        return W, status


def fp64_peak(blocks=148 * 8, threads=256, iters=20000, reps=5):
    """Measured FP64 FMA throughput (flop/s) of this GPU with the library's
    probe kernel, CUDA events on the current stream, best of ``reps``."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    fl = ctypes.c_double(0.0)
    best = 0.0
    for r in range(reps + 1):
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = lib().wc_fp64_peak_kernel(blocks, threads, iters, _ptr(sink), ctypes.byref(fl),
                                       _stream(s))
        e1.record(s)
        torch.cuda.synchronize()
        if st != 0:
            raise WcError(st, "fp64 peak probe")
        if r > 0:
            best = max(best, fl.value / (e0.elapsed_time(e1) * 1e-3))
    return best


def grid_barrier_check(skip_block=-1, rounds=100):
    """Runs the Q-map's grid barrier alone (see wc_grid_barrier_check);
    returns the status code (0 = WC_OK, 7 = WC_ERR_TIMEOUT)."""
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    return lib().wc_grid_barrier_check(_dptr(words), int(skip_block), int(rounds),
                                       _stream(torch.cuda.current_stream()))


def neighbour_barrier_check(skip_block=-1, span=1, rounds=100):
    """Runs the Q-map preconditioner's neighbour barrier alone (see
    wc_neighbour_barrier_check); returns the status code."""
    n = lib().wc_neighbour_barrier_words()
    words = torch.zeros(max(n, 8), dtype=torch.int32, device="cuda")
    return lib().wc_neighbour_barrier_check(_dptr(words), n, int(skip_block), int(span),
                                            int(rounds), _stream(torch.cuda.current_stream()))


def convert_f32(x):
    """The reduced-precision sweeps' binary64 -> binary32 -> binary64
    conversions applied to the float64 CUDA tensor ``x``: (f32, back)."""
    x = x.contiguous()
    f = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    back = torch.empty_like(x)
    st = lib().wc_convert_f32(_ptr(x), _dptr(f), _ptr(back), x.numel(),
                              _stream(torch.cuda.current_stream()))
    if st != 0:
        raise WcError(st, "convert_f32")
    return f, back


class Patches:
    """Batched independent cube patches (pooled state, one persistent launch
    per Runge-Kutta stage)."""

    def __init__(self, edges, gamma, pinf, D=None, pmin=None, flux="hll", precision="mixed",
                 energy_limiter=True, kmodel="allaire"):
        N = len(gamma)
        d = PatchesDesc()
        d.nphase = N
        D = list(D) if D is not None else [0.0] * N
        pmin = list(pmin) if pmin is not None else default_pmin(pinf)
        for p in range(N):
            d.gamma[p], d.pinf[p], d.D[p], d.pmin[p] = gamma[p], pinf[p], D[p], pmin[p]
        d.flux = FLUX[flux]
        d.precision = PREC[precision]
        d.energy_limiter = int(bool(energy_limiter))
        d.npatch = len(edges)
        d.kmodel = KMODEL[kmodel]
        self.edges = [int(e) for e in edges]
        arr = (ctypes.c_int * len(edges))(*self.edges)
        h = _VP()
        st = lib().wc_patches_init(ctypes.byref(d), arr, ctypes.byref(h))
        if st != 0:
            raise WcError(st, "wc_patches_init")
        self.h = h
        self.nv = 2 * N + 4
        self.ncell = lib().wc_patches_ncell(h)
        self.offsets = [lib().wc_patches_offset(h, p) for p in range(len(edges))]

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.wc_patches_destroy(h)
            self.h = None

    def _check(self, st):
        if st != 0:
            buf = ctypes.create_string_buffer(256)
            lib().wc_patches_last_error(self.h, buf, 256)
            raise WcError(st, buf.value.decode())

    def pack(self, states):
        """Pooled [NV][ncell] array (host numpy) from per-patch [NV][e][e][e]."""
        import numpy as np
        out = np.empty((self.nv, self.ncell))
        for p, S in enumerate(states):
            o = self.offsets[p]
            out[:, o:o + S[0].size] = S.reshape(self.nv, -1)
        return out

    def unpack(self, pooled, p):
        e = self.edges[p]
        o = self.offsets[p]
        return pooled[:, o:o + e ** 3].reshape(self.nv, e, e, e)

    def bind(self, U, stream=None, faces=True, prim=True):
        """Binds the pooled state with a new workspace; faces=False leaves out
        the face buffer (the window schedule's mixed sweep then runs in one
        pass), and with it prim=False the primitive slots (the window sweeps
        convert their cells then)."""
        b = lib().wc_patches_workspace_bytes(self.h)
        if not faces:
            b -= lib().wc_patches_face_buffer_bytes(self.h)
            if not prim:
                b -= lib().wc_patches_prim_buffer_bytes(self.h)
        n = (b + 7) // 8
        self.ws = torch.empty(n, dtype=torch.float64, device=U.device)
        self.U = U
        self._check(lib().wc_patches_set_state(self.h, _ptr(U), _ptr(self.ws), n * 8,
                                               _stream(stream)))
        return self

    def set_schedule(self, block, ctas_per_sm, dynamic):
        self._check(lib().wc_patches_set_schedule(self.h, block, ctas_per_sm, int(dynamic)))

    def rk_step(self, cfl=0.0, dt=0.0, nsteps=1, use_graph=False, stream=None):
        self._check(lib().wc_patches_rk_step(self.h, float(cfl), float(dt), int(nsteps),
                                             int(use_graph), _stream(stream)))

    def prim_to_cons(self, V, U=None, stream=None):
        U = torch.empty_like(V) if U is None else U
        self._check(lib().wc_patches_prim_to_cons(self.h, _ptr(V), _ptr(U), _stream(stream)))
        return U

    def rhs(self, U, L=None, stream=None):
        L = torch.empty_like(U) if L is None else L
        self._check(lib().wc_patches_rhs(self.h, _ptr(U), _ptr(L), _stream(stream)))
        return L

    def sync_status(self, stream=None):
        self._check(lib().wc_patches_sync_status(self.h, _stream(stream)))

    def autotune(self, cfl, steps=3, stream=None):
        b, c, d = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        ms = ctypes.c_double(0.0)
        self._check(lib().wc_patches_autotune(self.h, float(cfl), int(steps), _stream(stream),
                                              ctypes.byref(b), ctypes.byref(c),
                                              ctypes.byref(d), ctypes.byref(ms)))
        return {"block": b.value, "ctas_per_sm": c.value, "dynamic": d.value,
                "ms_per_step": ms.value}
