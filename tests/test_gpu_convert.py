"""The binary64 <-> binary32 conversions of the reduced-precision sweeps
(integer arithmetic on the IEEE 754 formats) against the hardware
conversions, bit for bit: random values over the whole binary32 range and
beyond, exact ties (round half to even), the largest binary32 and the values
that round past it to infinity, the normal/subnormal boundary, signed zeros,
infinities and NaN."""
import numpy as np
import pytest
import torch

from paper_2608_00746_b300 import wenoc

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(11)
    n = 1 << 20
    # random sign, exponent 2^-160 .. 2^160, random 52-bit fraction
    e = rng.integers(1023 - 160, 1023 + 160, size=n, dtype=np.int64)
    frac = rng.integers(0, 1 << 52, size=n, dtype=np.int64)
    sign = rng.integers(0, 2, size=n, dtype=np.int64) << 63
    bits = [sign | (e << 52) | frac]
    # ties: the 29 dropped bits exactly half, kept bits odd and even
    e2 = rng.integers(1023 - 126, 1023 + 128, size=4096, dtype=np.int64)
    kept = rng.integers(0, 1 << 23, size=4096, dtype=np.int64)
    for extra in (0x10000000, 0x0FFFFFFF, 0x10000001, 0, 0x1FFFFFFF):
        bits.append((e2 << 52) | (kept << 29) | extra)
        bits.append(np.int64(-0x8000000000000000) | (e2 << 52) | (kept << 29) | extra)
    x = np.concatenate([b.view(np.float64) for b in bits])
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, fmax, -fmax,
               np.nextafter(fmax, np.inf), fmax * (1 + 2.0 ** -24), fmax * (1 + 2.0 ** -25),
               fmax * (1 + 2.0 ** -24) * (1 - 2.0 ** -50), 2.0 ** 128, -2.0 ** 128,
               tiny, -tiny, np.nextafter(tiny, 0.0), tiny * (1 - 2.0 ** -25),
               tiny * (1 - 2.0 ** -24), tiny * 0.5, 2.0 ** -149, 2.0 ** -150, 1e-300, 1e300,
               5e-324, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52]
    # a sweep through every exponent of the normal/subnormal boundary region
    ks = np.arange(-160, 140, dtype=np.float64)
    walk = np.concatenate([2.0 ** ks * m for m in (1.0, 1.5, 1.9999999999, 1.00000006)])
    # binary64 subnormals and the values around half the smallest binary32
    # subnormal (2^-150), which round to zero or away from it
    sub = np.array([2.0 ** -1074, 2.0 ** -1030, 2.0 ** -151, 2.0 ** -150,
                    2.0 ** -150 * (1 + 2.0 ** -40), 2.0 ** -150 * (1 - 2.0 ** -40), 2.0 ** -149])
    return np.concatenate([x, np.array(special), walk, -walk, sub, -sub])


def test_conversions_match_hardware(gpu):
    x = torch.from_numpy(_cases()).cuda()
    f, back = wenoc.convert_f32(x)
    ref = x.float()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(f), nan)
    assert torch.equal(f[~nan].view(torch.int32), ref[~nan].view(torch.int32))
    refb = ref.double()
    assert torch.equal(back[~nan].view(torch.int64), refb[~nan].view(torch.int64))
    assert torch.isnan(back[nan]).all()


def test_empty_and_bad_arguments(gpu):
    x = torch.zeros(0, dtype=torch.float64, device="cuda")
    f, back = wenoc.convert_f32(x)
    assert f.numel() == 0 and back.numel() == 0
    assert wenoc.lib().wc_convert_f32(None, None, None, 5, None) != 0
