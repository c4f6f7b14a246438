"""FP64 CPU reference of the learned WENO-weight surrogate -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` leg may import this module.  It shares no code with the CUDA
path.

The paper has no learned component: the surrogate is a stand-in for the
WENO-W weights of Eq. 15 inside the coupled reconstruction of Eq. 16, so the
reading fixed here is the definition the GPU path is checked against:

* inputs per face side (stencil ordered towards the face) and phase p < 3:
  the five masses minus the cell's own, divided by the largest absolute such
  difference (0 when the stencil is flat), then the five fractions; unused
  phases and inputs 30, 31 are zero.  Eq. 15 depends only on ratios of the
  smoothness indicators, which are quadratic in f, so the weights of a
  stencil f and of a f + b (a != 0) coincide and the scaling loses nothing;
* network 32 -> 64 -> 64 -> 64 (ReLU) -> 16 (9 used), softmax over each
  phase's three outputs (the weights of the sub-stencils {i-2..i},
  {i-1..i+1}, {i..i+2});
* targets: the Eq. 15 weights of the masses on the same oriented stencil
  (ideal weights 0.1, 0.6, 0.3 for phases beyond N, which is what Eq. 15
  gives on an all-zero stencil);
* loss: the batch mean of the squared weight error summed over the 9
  outputs plus the squared errors those weights make in the normalised mass
  and fraction reconstructions (``loss_and_grads``); Adam (Kingma & Ba, beta1 0.9, beta2 0.999, eps 1e-8, bias
  corrected) on FP32 master parameters.

Features (``features``): the normalised mass differences formed in FP64
and every input rounded once to BF16.  The GPU stores features, weights,
hidden activations and the back-propagated deltas that enter a product in
BF16 and accumulates in FP32.  ``rounded=True``
reproduces those rounding points here (BF16 = round to nearest even of the
FP32 value) with every sum in FP64; ``rounded=False`` is the plain FP64
network, the one the finite-difference pins check.
"""
from __future__ import annotations

import numpy as np

from . import weno5_parts, wenow_weights

IN, H, OUT, NW = 32, 64, 16, 9
W1, W2 = 0, H * IN
W3 = W2 + H * H
W4 = W3 + H * H
NWEIGHT = W4 + OUT * H
B1, B2, B3, B4, NBIAS = 0, 64, 128, 192, 208
NPARAM = NWEIGHT + NBIAS
IDEAL = (0.1, 0.6, 0.3)


def bf16(x):
    """Round to BF16 (nearest even, via FP32) and return as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_round(x):
    """x (FP64) rounded once to BF16: 8 significant bits with the exponent
    range of binary32 (normal numbers from 2^-126, subnormal spacing
    2^-133), to nearest with ties to even.  Value-based: x = m 2^e with
    |m| in [1/2, 1) becomes a multiple of 2^max(e-8, -133).  (|x| < 2^128.)"""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    q = np.ldexp(1.0, np.maximum(e - 8, -133))
    return np.round(x / q) * q


def features(ms, als):
    """Inputs of rows of oriented stencils: ms, als [rows][P][5] (P <= 3
    phases, masses and fractions) -> [rows][32] (BF16 values as float64).

    Reading 18 as written: for each phase the differences d_k = f_k - f_i of
    the five masses to the cell's own (FP64), divided in FP64 by the largest
    |d_k| (all zero when that is 0: a flat stencil), then the five
    fractions; every value rounded once to BF16 (``bf16_round``)."""
    ms = np.asarray(ms, dtype=np.float64)
    als = np.asarray(als, dtype=np.float64)
    rows, P = ms.shape[0], ms.shape[1]
    X = np.zeros((rows, IN))
    for p in range(P):
        d = ms[:, p, :] - ms[:, p, 2:3]
        mx = np.max(np.abs(d), axis=1, keepdims=True)
        live = mx > 0.0
        q = np.where(live, d / np.where(live, mx, 1.0), 0.0)
        X[:, 10 * p:10 * p + 5] = bf16_round(q)
        X[:, 10 * p + 5:10 * p + 10] = bf16_round(als[:, p, :])
    return X


def targets(ms, N):
    """Plain Eq. 15 weights of each phase's oriented mass stencil, [rows][9].

    The smoothness indicators depend only on differences of the stencil
    values, so they are formed from f - f_i (the subtraction is exact for
    values within a factor two of f_i): on stencils whose variation is near
    the rounding of the values themselves, forming them from the raw values
    would leave the weights to rounding noise."""
    ms = np.asarray(ms, dtype=np.float64)
    rows = ms.shape[0]
    T = np.tile(np.array(IDEAL * 3), (rows, 1))
    for r in range(rows):
        for p in range(min(N, 3)):
            _, beta = weno5_parts(ms[r, p] - ms[r, p, 2])
            T[r, 3 * p:3 * p + 3] = wenow_weights(beta)
    return T


def unpack(flat, rounded=True):
    """Parameter dict from an FP32 array of NPARAM entries (weights rounded
    to BF16 as the parameter block stores them when rounded)."""
    flat = np.asarray(flat, dtype=np.float64)
    rw = bf16 if rounded else (lambda a: a)
    return {
        "W1": rw(flat[W1:W2].reshape(H, IN)), "W2": rw(flat[W2:W3].reshape(H, H)),
        "W3": rw(flat[W3:W4].reshape(H, H)), "W4": rw(flat[W4:NWEIGHT].reshape(OUT, H)),
        "b1": flat[NWEIGHT + B1:NWEIGHT + B2], "b2": flat[NWEIGHT + B2:NWEIGHT + B3],
        "b3": flat[NWEIGHT + B3:NWEIGHT + B4], "b4": flat[NWEIGHT + B4:NWEIGHT + NBIAS],
    }


def from_block(block):
    """Parameter dict from the raw bytes of the GPU parameter block."""
    block = np.asarray(block, dtype=np.uint8)
    w = block[:NWEIGHT * 2].view(np.uint16).astype(np.uint32) << 16
    wf = w.view(np.float32).astype(np.float64)
    b = block[NWEIGHT * 2:NWEIGHT * 2 + NBIAS * 4].view(np.float32).astype(np.float64)
    return unpack(np.concatenate([wf, b]), rounded=False)


def softmax3(z):
    y = np.empty((z.shape[0], NW))
    for p in range(3):
        a = z[:, 3 * p:3 * p + 3]
        e = np.exp(a - a.max(axis=1, keepdims=True))
        y[:, 3 * p:3 * p + 3] = e / e.sum(axis=1, keepdims=True)
    return y


def forward(P, X, rounded=True):
    """Weights [rows][9] and the activations (a0 = X, a1, a2, a3)."""
    r = bf16 if rounded else (lambda a: a)
    a0 = np.asarray(X, dtype=np.float64)
    a1 = r(np.maximum(a0 @ P["W1"].T + P["b1"], 0.0))
    a2 = r(np.maximum(a1 @ P["W2"].T + P["b2"], 0.0))
    a3 = r(np.maximum(a2 @ P["W3"].T + P["b3"], 0.0))
    z = a3 @ P["W4"].T + P["b4"]
    return softmax3(z), (a0, a1, a2, a3)


RECON_WEIGHT = 1.0


def candidates(X):
    """Candidate values of Eq. 10 (minus the cell value) at the face the
    stencil is ordered towards, for each phase's normalised masses and for
    its fractions shifted by the cell's fraction and divided by their largest
    absolute deviation (0 when that deviation is at most 1e-30): qm, qa
    [rows][3][3]."""
    X = np.asarray(X, dtype=np.float64)
    qm = np.zeros((X.shape[0], 3, 3))
    qa = np.zeros((X.shape[0], 3, 3))

    def cand(f):  # f [rows][5] with f[:, 2] = 0
        return np.stack([(2 * f[:, 0] - 7 * f[:, 1]) / 6, (2 * f[:, 3] - f[:, 1]) / 6,
                         (5 * f[:, 3] - f[:, 4]) / 6], axis=1)

    for p in range(3):
        xm = X[:, 10 * p:10 * p + 5]
        xa = X[:, 10 * p + 5:10 * p + 10]
        da = xa - xa[:, 2:3]
        mx = np.abs(da).max(axis=1, keepdims=True)
        big = mx > 1e-30    # smaller deviations count as flat
        da = np.where(big, da / np.where(big, mx, 1.0), 0.0)
        qm[:, p] = cand(xm)
        qa[:, p] = cand(da)
    return qm, qa


def loss_and_grads(P, X, T, rounded=True):
    """Loss and its gradient (a flat NPARAM array in the parameter order).
    Loss: the batch mean over samples of, summed over phases p,
    sum_s e_ps^2 + RECON_WEIGHT ((sum_s e_ps qm_ps)^2 + (sum_s e_ps qa_ps)^2)
    with e = y - T and qm, qa the candidates of ``candidates`` -- the weight
    error plus the error it makes in the two reconstructions that the
    acceptance test compares, in units of the stencil deviation."""
    r = bf16 if rounded else (lambda a: a)
    B = X.shape[0]
    y, (a0, a1, a2, a3) = forward(P, X, rounded)
    qm, qa = candidates(X)
    err = y - T
    loss = float(np.sum(err * err))
    dy = np.zeros_like(err)
    for p in range(3):
        s = slice(3 * p, 3 * p + 3)
        em = np.sum(err[:, s] * qm[:, p], axis=1, keepdims=True)
        ea = np.sum(err[:, s] * qa[:, p], axis=1, keepdims=True)
        loss += RECON_WEIGHT * float(np.sum(em * em + ea * ea))
        dy[:, s] = 2.0 * (err[:, s] + RECON_WEIGHT * (em * qm[:, p] + ea * qa[:, p])) / B
    loss /= B
    d = np.zeros((B, OUT))
    for p in range(3):
        s = slice(3 * p, 3 * p + 3)
        dot = np.sum(dy[:, s] * y[:, s], axis=1, keepdims=True)
        d[:, s] = y[:, s] * (dy[:, s] - dot)
    g = np.zeros(NPARAM)
    layers = [(a3, "W4", W4, NWEIGHT, B4), (a2, "W3", W3, W4, B3),
              (a1, "W2", W2, W3, B2), (a0, "W1", W1, W2, B1)]
    for k, (a_in, wname, w0, w1, b0) in enumerate(layers):
        out = P[wname].shape[0]
        g[NWEIGHT + b0:NWEIGHT + b0 + out] = d.sum(axis=0)
        dq = r(d)
        g[w0:w1] = (dq.T @ a_in).reshape(-1)
        if k < 3:
            da = dq @ P[wname]
            d = np.where(a_in > 0.0, da, 0.0)
    return loss, g


def adam(master, grads, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in FP64 (returns new master, m, v); padding stays zero."""
    m = b1 * m + (1.0 - b1) * grads
    v = b2 * v + (1.0 - b2) * grads * grads
    c1 = 1.0 / (1.0 - b1 ** step)
    c2 = 1.0 / (1.0 - b2 ** step)
    new = master - lr * (m * c1) / (np.sqrt(v * c2) + eps)
    new[padding_mask()] = 0.0
    return new, m, v


def padding_mask():
    mask = np.zeros(NPARAM, dtype=bool)
    mask[W1:W2] = (np.arange(W2 - W1) % IN) >= 30
    mask[W4:NWEIGHT] = ((np.arange(NWEIGHT - W4)) // H) >= NW
    mask[NWEIGHT + B4 + NW:] = True
    return mask


def oriented_stencils(U, N, direction, bc):
    """Oriented mass / fraction stencils of every cell of a state U [NV][...]
    (x fastest) in one direction: returns ms, als [2 ncell][min(N,3)][5] in
    row order 2 cell + side (side 0: f_{i-2..i+2}; side 1: mirrored).
    Boundary cells by index mapping: periodic wrap, reflective mirror,
    outflow copy of the edge cell (masses and fractions carry no sign)."""
    U = np.asarray(U, dtype=np.float64)
    nv = U.shape[0]
    P = min(N, 3)
    flat = U.reshape(nv, -1)
    ncell = flat.shape[1]
    shape = U.shape[1:]               # (nz, ny, nx) reversed axes
    axis = len(shape) - 1 - direction
    n = shape[axis]
    pos = np.indices(shape)[axis].reshape(-1)
    lo, hi = bc[2 * direction], bc[2 * direction + 1]

    def mapidx(j):
        j = np.array(j)
        out = j.copy()
        below, above = j < 0, j >= n
        if lo == "periodic":
            out = np.where(below, j % n, out)
        elif lo == "reflective":
            out = np.where(below, -1 - j, out)
        else:
            out = np.where(below, 0, out)
        if hi == "periodic":
            out = np.where(above, j % n, out)
        elif hi == "reflective":
            out = np.where(above, 2 * n - 1 - j, out)
        else:
            out = np.where(above, n - 1, out)
        return out

    ms = np.zeros((2 * ncell, P, 5))
    als = np.zeros((2 * ncell, P, 5))
    for s in range(5):
        jj = mapidx(pos - 2 + s)
        idx = np.moveaxis(np.indices(shape), 0, -1).reshape(-1, len(shape)).copy()
        idx[:, axis] = jj
        src = np.ravel_multi_index(tuple(idx.T), shape)
        for p in range(P):
            mv = flat[p, src]
            av = flat[nv - N + p, src]
            ms[0::2, p, s] = mv
            als[0::2, p, s] = av
            ms[1::2, p, 4 - s] = mv
            als[1::2, p, 4 - s] = av
    return ms, als
