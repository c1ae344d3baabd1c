"""The helpers that take compares, conversions and divisions off the FP64 pipe,
against the hardware's own instructions on the same inputs: the integer
float -> double must equal the conversion instruction bit for bit (every
class of float: zeros, subnormals, normals, infinities, NaNs), the integer
predicates must agree with the IEEE compares everywhere on their stated
domain, the integer double -> float must equal the conversion instruction bit
for bit, the embedded difference of the mixed trial must agree with FP64, and
the reciprocal must lie within one ulp of the IEEE division."""
import numpy as np
import pytest

from paper_2511_21031_gb300 import pab

pytestmark = pytest.mark.gpu


def _floats(rng, n):
    specials = np.array([0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x007fffff, 0x807fffff,
                         0x00800000, 0x80800000, 0x7f7fffff, 0xff7fffff, 0x7f800000, 0xff800000,
                         0x7fc00000, 0xffc00000, 0x7fc12345, 0x3f800000, 0x00400000, 0x00000100],
                        dtype=np.uint32)
    every_class = rng.integers(0, 2**32, size=n // 2, dtype=np.uint64).astype(np.uint32)
    subnormal = rng.integers(1, 2**23, size=n // 8, dtype=np.uint64).astype(np.uint32)
    subnormal |= (rng.integers(0, 2, size=subnormal.size) << 31).astype(np.uint32)
    values = rng.normal(size=n - specials.size - every_class.size - subnormal.size)
    values = (values * 10.0 ** rng.uniform(-12, 3, size=values.size)).astype(np.float32)
    return np.concatenate([specials.view(np.float32), every_class.view(np.float32),
                           subnormal.view(np.float32), values])


def _doubles(rng, n):
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324,
                         2.2250738585072014e-308, 1.7976931348623157e308, 1.0, -1.0, 1e-30,
                         3e38, 0.2, 5.0], dtype=np.float64)
    # exact ties between neighbouring floats (rounded to even), one ulp either side of
    # them, and the overflow edge of the largest float
    f = (10.0 ** rng.uniform(-37, 38, size=n // 16)).astype(np.float32).astype(np.float64)
    half = np.spacing(f.astype(np.float32)).astype(np.float64) / 2
    ties = np.concatenate([f + half, f + half * (1 + 2.0 ** -40), f + half * (1 - 2.0 ** -40)])
    fmax = float(np.finfo(np.float32).max)
    hmax = 2.0 ** 103  # half an ulp of the largest float (ulp 2^104)
    edge = np.array([fmax, fmax + hmax, fmax + hmax * (1 - 2.0 ** -40), 2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -30)])
    mag = 10.0 ** rng.uniform(-300, 300, size=n - specials.size - ties.size - edge.size)
    near = rng.random(mag.size) < 0.5
    mag[near] = 10.0 ** rng.uniform(-12, 4, size=int(near.sum()))
    mag = np.concatenate([ties, edge, mag])
    sign = np.where(rng.random(mag.size) < 0.3, -1.0, 1.0)
    return np.concatenate([specials, sign * mag])


def test_bit_helpers_match_the_hardware():
    import torch
    rng = np.random.default_rng(77)
    n = 1 << 18
    f = _floats(rng, n)
    x = _doubles(rng, n)
    y = np.abs(_doubles(rng, n))
    y[~np.isfinite(y)] = 1.0
    tie = rng.random(n) < 0.2  # x == y and |x| == y exactly
    y[tie & np.isfinite(x)] = np.abs(x[tie & np.isfinite(x)])
    y[: 16] = 0.0
    out = pab.pab_bits_check(torch.as_tensor(f, device="cuda"), torch.as_tensor(x, device="cuda"),
                             torch.as_tensor(y, device="cuda"))
    o = {k: v.cpu().numpy() for k, v in out.items()}

    nan = np.isnan(f)
    np.testing.assert_array_equal(o["f2d"][~nan].view(np.uint64), o["f2d_hw"][~nan].view(np.uint64))
    np.testing.assert_array_equal(o["f2d"][~nan].view(np.uint64),
                                  f[~nan].astype(np.float64).view(np.uint64))
    assert np.all(np.isnan(o["f2d"][nan]))
    assert np.count_nonzero(o["cmp"]) == 0, np.unique(o["cmp"], return_counts=True)

    ax = np.abs(x)
    dom = np.isfinite(x) & (ax >= 2.0 ** -1020) & (ax <= 2.0 ** 1020)
    div, rcp, seed = o["div"][dom], o["rcp"][dom], o["seed"][dom]
    np.testing.assert_array_equal(div, 1.0 / x[dom])  # the IEEE division, as numpy's
    ulp = np.spacing(np.abs(div))
    err_ulp = np.abs(rcp - div) / ulp
    seed_rel = np.abs(seed.astype(np.longdouble) * x[dom].astype(np.longdouble) - 1)
    print(f"reciprocal: max {err_ulp.max():.2f} ulp, {np.mean(err_ulp == 0):.5f} exact; "
          f"seed max relative error 2^{np.log2(float(seed_rel.max())):.2f}")
    assert err_ulp.max() <= 1.0
    assert np.mean(err_ulp == 0) > 0.99
    assert float(seed_rel.max()) < 2.0 ** -18  # the correction's truncation e0^3 < 2^-54
    bad = ~np.isfinite(x) | (x == 0)
    assert np.all(np.isnan(o["rcp"][bad]))


def _near_ties(rng, base, n):
    """base (1 + delta) with delta at every scale from 2^-60 to 1/2, either sign, and zero."""
    k = rng.integers(8, 61, size=n)
    delta = np.where(rng.random(n) < 0.8, np.ldexp(1.0, -k) * rng.choice([-1.0, 1.0], size=n),
                     rng.uniform(-0.5, 0.5, size=n))
    delta[rng.random(n) < 0.05] = 0.0
    return base * (1.0 + delta)


@pytest.mark.parametrize("tol", [1e-4, 1e-7, 1e-8, 0.3])
def test_bracketed_accept_tests_decide_as_the_exact_ones(tol):
    """The FP64 trial's accept test decided by its FP32 error estimate outside tol (1 -/+ 2^-16),
    and the mixed trial's component test decided by an FP32 bound on the TwoSum parts outside
    T (1 -/+ 2^-20), give the exact FP64 tests' decisions on inputs crowded at the tolerance
    (relative offsets from 2^-60 to 1/2), at every magnitude, and on the edges (zeros,
    magnitudes outside the bracket's range, infinities, NaNs)."""
    import torch
    rng = np.random.default_rng(31)
    n = 1 << 21
    v_floor = 1e-3 * np.sqrt(101325.0 / 1000.0)
    tol3 = 3.0 * tol
    R = 10.0 ** rng.uniform(-9, -2, size=n)
    V = rng.normal(size=n) * 10.0 ** rng.uniform(-4, 3, size=n)
    V[rng.random(n) < 0.05] = 0.0
    vs = np.maximum(np.abs(V), v_floor)
    eR = _near_ties(rng, tol3 * R, n) * rng.choice([-1.0, 1.0], size=n)
    eV = _near_ties(rng, tol3 * vs, n) * rng.choice([-1.0, 1.0], size=n)
    # one component clearly inside for half of them, so that the other decides
    inside = rng.random(n) < 0.5
    eR[inside] *= 0.25
    eV[~inside & (rng.random(n) < 0.5)] *= 0.25
    edge = rng.random(n) < 0.02
    R[edge] = rng.choice([1e-40, 1e-31, 1e31, 1e40], size=edge.sum())
    eR[edge] = tol3 * R[edge] * rng.choice([0.5, 1.0, 2.0], size=edge.sum())
    odd = rng.choice(n, 64, replace=False)
    eR[odd[:16]] = np.inf
    eR[odd[16:32]] = np.nan
    eV[odd[32:48]] = 0.0
    eR[odd[48:]] = 1e300
    trial = np.stack([R, V, eR, eV], axis=1)

    k1 = (rng.normal(size=n) * 10.0 ** rng.uniform(-12, 0, size=n)).astype(np.float32)
    k2 = np.where(rng.random(n) < 0.5, k1 * (1 + rng.normal(size=n) * 1e-3),
                  rng.normal(size=n) * 10.0 ** rng.uniform(-12, 0, size=n)).astype(np.float32)
    half = (k1.astype(np.float64) + k2.astype(np.float64)) / 2
    k3 = _near_ties(rng, half, n).astype(np.float32)          # cancellation in 2 k3 - (k1 + k2)
    D = 2.0 * k3.astype(np.float64) - (k1.astype(np.float64) + k2.astype(np.float64))
    T = np.abs(_near_ties(rng, D, n)).astype(np.float32)
    T[rng.random(n) < 0.01] = 0.0
    kk = np.stack([k1, k2, k3, T], axis=1)
    kk[odd[:16], 3] = np.inf
    kk[odd[16:32], 0] = np.nan
    kk[odd[32:48], 2] = np.inf
    kk[odd[48:], 3] = np.float32(1e-45)

    out = pab.pab_accept_check(torch.as_tensor(trial, device="cuda"),
                               torch.as_tensor(np.ascontiguousarray(kk), device="cuda"), tol,
                               v_floor).cpu().numpy()
    bad64 = np.flatnonzero(out[:, 0] != out[:, 1])
    bad32 = np.flatnonzero(out[:, 2] != out[:, 3])
    assert bad64.size == 0, trial[bad64[:5]]
    assert bad32.size == 0, kk[bad32[:5]]
    # the inputs straddle the tolerance: both decisions occur in quantity
    assert 0.2 < out[:, 1].mean() < 0.8 and 0.2 < out[:, 3].mean() < 0.8
