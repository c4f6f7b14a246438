"""Operation counts of the oracle (TEST INFRASTRUCTURE, and the source of the
algorithmic flop counts of the roofline).

``wenoc_oracle.c`` compiled as C++ with -DOR_COUNT and ``op_count.hpp``
(liboracle_count.so) counts every floating-point operation it performs,
attributed to the step it belongs to: cons -> prim (Eq. 27), smoothness
indicators and candidates (Eq. 11), weights (Eq. 15), the combination
(Eq. 10), the limiter chain (Eq. 17-21), V -> U, the Riemann flux with u-hat,
the conservative update (Eq. 3) and the Runge-Kutta stage.  One rhs
evaluation on a smooth periodic state (every limiter factor 1: the common
path) is counted.

The per-cell-direction count takes each step as often as the method needs it
per cell and direction: one cons -> prim (the oracle converts each of the
five stencil cells of every cell), smoothness indicators of the N masses, the
D velocity components and the pressure once (the fractions use the masses'
weights, and the mirrored stencil of the other face has the same three
values), candidates of all 2N + D + 1 variables on both faces, and the
weights, combinations, limiter chain, flux and update as the oracle does
them; the Runge-Kutta stage is shared by the D sweeps of a stage.
Material constants the oracle recomputes per call (A_p, B_p of Eq. 26) are
not counted.  Flops: add/subtract, multiply, divide and square root are 1
each (the oracle forms no fused multiply-adds); comparisons are 0.

  python -m oracle.op_count      # rewrites paper_2608_00746_b300/op_counts.json
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess

import numpy as np

from . import Grid, _Grid, prim_to_cons

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wenoc_oracle.c")
_HDR = os.path.join(_HERE, "op_count.hpp")
_LIB = os.path.join(_HERE, "liboracle_count.so")
OUT = os.path.join(os.path.dirname(_HERE), "paper_2608_00746_b300", "op_counts.json")

CATS = ["other", "prim", "beta", "cand", "weights", "combine", "limit", "v2u", "flux",
        "update", "rk", "const", "recon"]
KINDS = ["add", "mul", "div", "sqrt", "cmp", "calls"]
CASES = [(2, 1, "hllc"), (2, 2, "hll"), (2, 2, "hllc"), (3, 2, "hll"), (3, 3, "hll"),
         (5, 2, "hllc")]
# the steps the mixed-precision form keeps in FP64 (pressure recovery, the
# limiter's factors and normalisation with the face states they act on,
# the update and accumulation); the rest runs in FP32
FP64_STEPS = ("prim", "limit", "v2u", "update", "rk")


def build(force=False):
    if force or not os.path.exists(_LIB) or any(
            os.path.getmtime(_LIB) < os.path.getmtime(f) for f in (_SRC, _HDR)):
        cmd = ["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-DOR_COUNT", "-include", _HDR, "-x", "c++", _SRC,
               "-o", _LIB]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        gp = ctypes.POINTER(_Grid)
        _lib.or_rhs.argtypes = [gp, dp, dp]
        _lib.or_rhs.restype = ctypes.c_int
        _lib.or_rk_stage.argtypes = [gp, ctypes.c_double, dp, ctypes.c_double, dp,
                                     ctypes.c_double, ctypes.c_double, dp, dp]
        _lib.or_rk_stage.restype = None
        _lib.or_op_counts_read.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        _lib.or_op_counts_reset.argtypes = []
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _read():
    out = np.zeros(len(CATS) * len(KINDS), dtype=np.int64)
    lib().or_op_counts_read(out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return out.reshape(len(CATS), len(KINDS)).astype(np.float64)


def smooth_state(N, D, n):
    """A smooth periodic state with every phase present: fractions in about
    [0.1, 0.6], densities 1 to 1000, small smooth velocity and pressure
    variations (no limiter acts)."""
    shape = (n,) * D
    x = np.meshgrid(*[(np.arange(n) + 0.5) / n for _ in range(D)], indexing="ij")
    x = [xi.T for xi in x]  # [nz][ny][nx] order
    s = sum(x)
    raw = [1.0 + 0.4 * np.sin(2 * np.pi * (s + p / N)) for p in range(N)]
    tot = sum(raw)
    alpha = [r / tot for r in raw]
    rho = [10.0 ** (3.0 * p / max(N - 1, 1)) for p in range(N)]
    V = np.zeros((2 * N + D + 1,) + alpha[0].shape)
    for p in range(N):
        V[p] = alpha[p] * rho[p]
        V[N + D + 1 + p] = alpha[p]
    for j in range(D):
        V[N + j] = 0.1 * (1 + j) * np.sin(2 * np.pi * (x[j] + 0.1))
    V[N + D] = 1e5 * (1.0 + 0.1 * np.cos(2 * np.pi * s))
    gam = [1.4, 4.4, 6.1, 1.67, 2.0][:N]
    pinf = [0.0, 6e8, 2e9, 0.0, 1e8][:N]
    return shape, gam, pinf, V


def count(N, D, flux, n=None):
    """Per-cell-direction operation counts of the common path (see the
    module's docstring), per step, plus the flop total and its FP64 / FP32
    split in the mixed-precision form."""
    n = n or {1: 64, 2: 24, 3: 12}[D]
    shape, gam, pinf, V = smooth_state(N, D, n)
    g = Grid(tuple(reversed(shape)) if D > 1 else shape, (1.0 / n,) * D, gam, pinf, flux=flux)
    U = np.ascontiguousarray(prim_to_cons(g, V))
    L = np.zeros_like(U)
    lib().or_op_counts_reset()
    rc = lib().or_rhs(g.ref(), _p(U), _p(L))
    if rc != 0:
        raise RuntimeError(f"counting rhs returned {rc}")
    c_rhs = _read()
    lib().or_op_counts_reset()
    out = np.empty_like(U)
    lib().or_rk_stage(g.ref(), 0.75, _p(U), 0.25, _p(U), 0.25, 1e-6, _p(L), _p(out))
    c_rk = _read()
    cells = U[0].size
    NV = 2 * N + D + 1
    flops = {}
    cat = {c: i for i, c in enumerate(CATS)}

    def fl(c, src):
        return src[cat[c], 0] + src[cat[c], 1] + src[cat[c], 2] + src[cat[c], 3]

    def per_call(c, src=c_rhs):
        return fl(c, src) / max(src[cat[c], 5], 1)

    recon = c_rhs[cat["recon"], 5]
    flops["prim"] = per_call("prim")
    flops["beta"] = per_call("beta") * (N + D + 1)
    flops["cand"] = per_call("cand") * 2 * NV
    for c in ("weights", "combine", "limit", "v2u"):
        flops[c] = fl(c, c_rhs) / recon
    flops["flux"] = per_call("flux")
    flops["update"] = per_call("update")
    flops["rk"] = fl("rk", c_rk) / cells / D
    total = sum(flops.values())
    fp64 = sum(flops[c] for c in FP64_STEPS)
    return {"N": N, "D": D, "flux": flux, "grid": list(shape),
            "flops_per_cell_dir": round(total, 2),
            "flops_per_cell_dir_by_step": {k: round(v, 2) for k, v in flops.items()},
            "mixed_fp64_flops_per_cell_dir": round(fp64, 2),
            "mixed_fp32_flops_per_cell_dir": round(total - fp64, 2),
            "oracle_flops_per_cell_dir_literal": round(
                sum(fl(c, c_rhs) for c in CATS if c != "const") / (cells * D)
                + flops["rk"], 2)}


def main():
    res = {"note": "written by python -m oracle.op_count from the oracle's counting build; "
                   "per interior cell and direction sweep, common path",
           "fp64_steps_in_mixed": list(FP64_STEPS),
           "counts": [count(N, D, f) for N, D, f in CASES]}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1)
        fh.write("\n")
    for c in res["counts"]:
        print(c["N"], c["D"], c["flux"], c["flops_per_cell_dir"], c["flops_per_cell_dir_by_step"])


if __name__ == "__main__":
    main()
