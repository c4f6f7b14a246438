"""Pins of the FP64 surrogate reference (oracle/mlp.py) against what
mathematics fixes: finite differences of the loss, the closed form of a
uniform softmax, BF16 round-to-nearest-even ties, Adam's first step, the
affine invariance of the WENO-W weights the features rely on (Eq. 15),
textbook weight values on linear and step stencils, and a brute-force
stencil gather."""
import numpy as np

import oracle
from oracle import mlp


def _flat(P):
    return np.concatenate([P[k].reshape(-1) for k in ("W1", "W2", "W3", "W4")] +
                          [P[k] for k in ("b1", "b2", "b3", "b4")])


def _random_params(rng, scale=0.3):
    flat = rng.normal(size=mlp.NPARAM) * scale
    flat[mlp.padding_mask()] = 0.0
    return mlp.unpack(flat, rounded=False)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    P = _random_params(rng)
    X = rng.normal(size=(24, 32))
    X[:, 30:] = 0.0
    T = rng.random((24, 9))
    L, g = mlp.loss_and_grads(P, X, T, rounded=False)
    flat = _flat(P)
    h = 1e-6
    picks = np.concatenate([rng.choice(mlp.NPARAM, 300, replace=False),
                            np.arange(mlp.NWEIGHT, mlp.NPARAM, 7)])
    for i in picks:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unpack(fp, False), X, T, False)
        lm, _ = mlp.loss_and_grads(mlp.unpack(fm, False), X, T, False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 2e-9 + 1e-6 * abs(g[i]), (i, fd, g[i])
    # a mistake in any layer shows up as a gradient of the wrong size
    assert np.abs(g[mlp.W1:mlp.W2]).max() > 1e-4
    assert np.abs(g[mlp.W4:mlp.NWEIGHT]).max() > 1e-4


def test_uniform_softmax_closed_form():
    """W4 = 0, b4 = 0: every weight is 1/3, loss = mean sum (1/3 - T)^2, and
    the logit gradient is (1/3)(dy - mean dy) per phase."""
    rng = np.random.default_rng(1)
    flat = rng.normal(size=mlp.NPARAM) * 0.3
    flat[mlp.W4:mlp.NWEIGHT] = 0.0
    flat[mlp.NWEIGHT + mlp.B4:] = 0.0
    P = mlp.unpack(flat, rounded=False)
    X = rng.normal(size=(8, 32))
    T = rng.random((8, 9))
    y, _ = mlp.forward(P, X, rounded=False)
    assert np.allclose(y, 1.0 / 3.0, rtol=0, atol=1e-15)
    # the reconstruction term: every candidate (Eq. 10) reproduces a linear
    # stencil, slope 1/2 per cell, at the face half a cell away: q = 1/4
    lin = np.zeros((1, 32))
    lin[0, 0:5] = [-1.0, -0.5, 0.0, 0.5, 1.0]
    qm, qa = mlp.candidates(lin)
    assert np.allclose(qm[0, 0], [0.25, 0.25, 0.25], atol=1e-15)
    assert np.all(qa == 0.0) and np.all(qm[0, 1:] == 0.0)
    X[:, 30:] = 0.0
    Xf = X.copy()
    for p in range(3):   # flat stencils: no reconstruction term
        Xf[:, 10 * p:10 * p + 10] = 0.0
    L, g = mlp.loss_and_grads(P, Xf, T, rounded=False)
    assert abs(L - np.sum((1.0 / 3.0 - T) ** 2) / 8) < 1e-14
    dy = 2.0 * (1.0 / 3.0 - T) / 8
    db4 = np.zeros(16)
    for p in range(3):
        s = slice(3 * p, 3 * p + 3)
        db4[s] = (dy[:, s] - dy[:, s].mean(axis=1, keepdims=True)).sum(axis=0) / 3.0
    assert np.allclose(g[mlp.NWEIGHT + mlp.B4:], db4, rtol=0, atol=1e-15)


def test_bf16_round_to_nearest_even():
    u = 2.0 ** -7  # BF16 spacing on [1, 2)
    assert mlp.bf16(1.0 + u / 2) == 1.0             # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3 * u / 2) == 1.0 + 2 * u  # tie -> even (1 + 2u)
    assert mlp.bf16(1.0 + 0.51 * u) == 1.0 + u
    assert mlp.bf16(-3.0) == -3.0
    assert mlp.bf16(0.0) == 0.0


def _all_bf16_values():
    """Every finite BF16 value (all 16-bit patterns but Inf/NaN), sorted,
    with the parity of its last significand bit."""
    pat = np.arange(1 << 16, dtype=np.uint32)
    pat = pat[(pat & 0x7F80) != 0x7F80]
    v = (pat << 16).view(np.float32).astype(np.float64)
    order = np.argsort(v, kind="stable")
    v, pat = v[order], pat[order]
    keep = np.concatenate([[True], v[1:] != v[:-1]])   # +0 / -0
    return v[keep], (pat[keep] & 1) == 0


def test_bf16_round_is_the_nearest_bf16_value():
    """bf16_round against brute force over the whole BF16 value set: the
    nearest value, ties to the one with an even last bit; values inside the
    subnormal range and exact ties included."""
    vals, even = _all_bf16_values()
    rng = np.random.default_rng(5)
    x = np.concatenate([
        rng.standard_normal(3000) * 10.0 ** rng.integers(-6, 6, 3000),
        rng.random(500) * 2.0 ** -126,                       # subnormal BF16 range
        rng.random(200) * 2.0 ** -133,                       # below the smallest
        vals[(vals > -1e30) & (vals < 1e30)][::97],          # representable values
    ])
    mids = 0.5 * (vals[1:] + vals[:-1])
    x = np.concatenate([x, mids[np.abs(mids) < 1e30][::61]])   # exact ties
    j = np.clip(np.searchsorted(vals, x), 1, len(vals) - 1)
    lo, hi = vals[j - 1], vals[j]
    dlo, dhi = x - lo, hi - x
    pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(even[j - 1], lo, hi)))
    got = mlp.bf16_round(x)
    assert np.array_equal(got, pick)
    u = 2.0 ** -7
    assert mlp.bf16_round(1.0 + u / 2) == 1.0
    # just above a tie rounds up; rounding through FP32 first would land on
    # the tie and round down
    x = 1.0 + u / 2 + 2.0 ** -40
    assert mlp.bf16_round(x) == 1.0 + u and mlp.bf16(x) == 1.0
    assert mlp.bf16_round(2.0 ** -134) == 0.0 and mlp.bf16_round(1.5 * 2.0 ** -133) == 2.0 ** -132


def test_features_hand_computed_stencil():
    """Masses 1, 2, 4, 7, 5 around the cell value 4: differences -3, -2, 0,
    3, 1 over the largest, 3, are -1, -2/3, 0, 1, 1/3; to 8 significant
    bits 2/3 = 0.10101010|10..b rounds up to 171/256 and 1/3 to 171/512."""
    ms = np.zeros((1, 3, 5))
    ms[0, 0] = [1.0, 2.0, 4.0, 7.0, 5.0]
    al = np.zeros((1, 3, 5))
    al[0, 0] = [0.0, 0.1, 0.5, 0.9, 1.0]
    X = mlp.features(ms, al)
    assert X[0, 0:5].tolist() == [-1.0, -171.0 / 256.0, 0.0, 1.0, 171.0 / 512.0]
    # 0.1 = 1.1001100|1100..b x 2^-4 -> 1.1001101b x 2^-4 = 205/2048; 0.9 =
    # 1.1100110|0110..b x 2^-1 -> 1.1100110b x 2^-1 = 115/128
    assert X[0, 5:10].tolist() == [0.0, 205.0 / 2048.0, 0.5, 115.0 / 128.0, 1.0]
    assert np.all(X[0, 10:] == 0.0)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    master = rng.normal(size=mlp.NPARAM)
    master[mlp.padding_mask()] = 0.0
    g = rng.normal(size=mlp.NPARAM)
    new, m, v = mlp.adam(master, g, np.zeros_like(g), np.zeros_like(g), 1e-3, 1)
    keep = ~mlp.padding_mask()
    expect = master - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(new[keep], expect[keep], rtol=0, atol=1e-15)
    assert np.all(new[~keep] == 0.0)


def test_features_affine_invariance_and_flat_stencil():
    rng = np.random.default_rng(3)
    ms = rng.random((50, 3, 5)) * 100
    al = rng.random((50, 3, 5))
    X = mlp.features(ms, al)
    assert np.array_equal(mlp.features(ms * 8.0, al), X)         # power-of-two scaling
    assert np.array_equal(mlp.features(-ms, al)[:, 0:5], -X[:, 0:5])  # sign symmetry
    assert np.all(np.abs(X[:, [0, 1, 3, 4, 10, 11, 13, 14]]) <= 1.0)
    assert np.all(X[:, [2, 12, 22]] == 0.0)
    assert np.all(X[:, 30:] == 0.0)
    assert np.array_equal(X[:, 5:10], mlp.bf16_round(al[:, 0, :]))
    flat = np.full((1, 3, 5), 7.5)
    Xf = mlp.features(flat, np.full((1, 3, 5), 0.25))
    assert np.all(Xf[0, [0, 1, 2, 3, 4]] == 0.0)
    # the plain weights the features stand for are affine invariant (Eq. 15)
    f = rng.random(5)
    w0 = oracle.wenow_weights(oracle.weno5_parts(f)[1])
    w1 = oracle.wenow_weights(oracle.weno5_parts(3.0 * f - 11.0)[1])
    assert np.allclose(w0, w1, rtol=1e-12, atol=1e-14)


def test_targets_textbook_stencils():
    lin = np.array([[[0.0, 1.0, 2.0, 3.0, 4.0]] * 3])
    assert np.allclose(mlp.targets(lin, 3), [0.1, 0.6, 0.3] * 3, atol=1e-15)
    step = np.zeros((1, 3, 5))
    step[0, 0] = [0.0, 0.0, 0.0, 1.0, 1.0]   # discontinuity right of the cell
    T = mlp.targets(step, 1)
    assert np.allclose(T[0, :3], [1.0, 0.0, 0.0], atol=1e-15)
    assert np.allclose(T[0, 3:], [0.1, 0.6, 0.3] * 2, atol=1e-15)  # phases beyond N
    # a flat stencil: all indicators zero, Eq. 15 gives the ideal weights
    assert np.allclose(mlp.targets(np.ones((1, 3, 5)), 3), [0.1, 0.6, 0.3] * 3, atol=1e-15)


def test_oriented_stencils_brute_force():
    rng = np.random.default_rng(4)
    N, nx, ny = 3, 7, 5
    U = rng.random((2 * N + 3, ny, nx))
    bcs = {0: ("reflective", "outflow"), 1: ("periodic", "periodic")}
    for d in (0, 1):
        bc = (bcs[0][0], bcs[0][1], bcs[1][0], bcs[1][1], "periodic", "periodic")
        if d == 1:
            bc = ("periodic", "periodic", "reflective", "outflow", "periodic", "periodic")
        ms, al = mlp.oriented_stencils(U, N, d, bc)
        n = nx if d == 0 else ny
        lo, hi = bc[2 * d], bc[2 * d + 1]
        for j in range(ny):
            for i in range(nx):
                cell = j * nx + i
                pos = i if d == 0 else j
                vals = []
                for s in range(5):
                    q = pos - 2 + s
                    if q < 0:
                        q = {"periodic": q + n, "reflective": -1 - q, "outflow": 0}[lo]
                    elif q >= n:
                        q = {"periodic": q - n, "reflective": 2 * n - 1 - q,
                             "outflow": n - 1}[hi]
                    vals.append((j, q) if d == 0 else (q, i))
                for p in range(N):
                    m = [U[p, a, b] for a, b in vals]
                    f = [U[2 * N + 3 - N + p, a, b] for a, b in vals]
                    assert np.array_equal(ms[2 * cell, p], m)
                    assert np.array_equal(ms[2 * cell + 1, p], m[::-1])
                    assert np.array_equal(al[2 * cell, p], f)
                    assert np.array_equal(al[2 * cell + 1, p], f[::-1])
