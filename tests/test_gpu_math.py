"""The library's FP64 shortcuts against high-precision references (numpy long
double on the host): the binomial series of the gas term, around an exact base
or around the nearest node of the handle's table (degree 11, used only where
its truncation is below half an ulp), must be no less accurate than CUDA's
exp(a log(x)) it replaces."""
import numpy as np
import pytest

from paper_2511_21031_gb300 import pab

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.mark.parametrize("a", [3.0, 4.2, 5.0])
def test_gas_series_as_accurate_as_exp_log(a):
    import torch
    g = np.random.default_rng(60)
    n = 200_000
    Rb = np.exp(g.uniform(np.log(0.05), np.log(20.0), size=n))
    d = g.uniform(-0.05, 0.05, size=n)                 # beyond the series range too
    R = Rb * (1.0 + d)
    gas, gtab, exact = pab.pab_math_check(torch.as_tensor(R, device="cuda"),
                                             torch.as_tensor(Rb, device="cuda"), a)
    ref = np.power(1.0 / R.astype(np.longdouble), np.longdouble(a))
    e_series = np.abs(gas.cpu().numpy().astype(np.longdouble) - ref) / ref
    e_explog = np.abs(exact.cpu().numpy().astype(np.longdouble) - ref) / ref
    e_table = np.abs(gtab.cpu().numpy().astype(np.longdouble) - ref) / ref
    assert float(e_series.max()) <= float(e_explog.max()) + 4 * ULP
    assert float(e_series.max()) <= 24 * ULP
    # the node table (used by handles) is a pure function of R and at least as accurate
    assert float(e_table.max()) <= float(e_explog.max()) + 4 * ULP
    assert float(e_table.max()) <= 16 * ULP
    small = np.abs(d) < 0.005
    assert small.sum() > 10000
    # where the series is used the error stays at the base value's error plus a few ulp
    ref_b = np.power(1.0 / Rb.astype(np.longdouble), np.longdouble(a))
    assert float(np.median(e_series[small])) <= 4 * ULP
    del ref_b


@pytest.mark.parametrize("gamma", [1.0, 1.4, 5.0 / 3.0])
def test_fp32_gas_term_within_its_bound(gamma):
    """(1 + u)^(-3 gamma) - 1 in FP32 against FP64, in ulps of the FP32 result: the
    branch-free evaluation of the mixed right-hand side stays within the bound its
    header states, and near the library composition expm1f(-a log1pf(u))."""
    import torch
    a = np.float32(3.0 * gamma)
    rng = np.random.default_rng(5)
    near = np.concatenate([10.0 ** rng.uniform(-12, np.log10(0.5), 200000),
                           -(10.0 ** rng.uniform(-12, np.log10(0.5), 200000))])
    wide = np.concatenate([rng.uniform(-0.8, 0.0, 100000), 10.0 ** rng.uniform(-0.3, 3, 100000)])
    for u, bound in ((near, 8.0), (wide, 16.0)):
        u32 = np.concatenate([u, [0.0, -0.0]]).astype(np.float32)
        out, lib = pab.pab_gas32_check(torch.as_tensor(u32, device="cuda"), float(a))
        out, lib = out.cpu().numpy().astype(np.float64), lib.cpu().numpy().astype(np.float64)
        exact = np.expm1(-float(a) * np.log1p(u32.astype(np.float64)))
        ulp = np.spacing(np.abs(exact.astype(np.float32))).astype(np.float64)
        ulp[exact == 0] = np.finfo(np.float32).smallest_subnormal
        e_new = np.abs(out - exact) / ulp
        e_lib = np.abs(lib - exact) / ulp
        print(f"gamma {gamma}: max {e_new.max():.2f} ulp (CUDA expm1f/log1pf: {e_lib.max():.2f})")
        assert np.all(np.isfinite(out))
        assert e_new.max() <= bound
        assert e_new.max() <= 1.5 * e_lib.max() + 2.0
        assert np.all(out[u32 == 0] == 0)


def test_table_driven_exp_within_two_ulp():
    """The Euler-Lagrange smear's FP64 e^x (Tang's table-driven method, 32 entries, degree-6
    Taylor polynomial) against a long-double reference: within 2^-51 relative (2 ulp at the
    bottom of a binade) on the smear's range [-20, 1], on the reduction's edges (x = (k + 1/2)
    ln2/32, where |r| is largest, and x near every multiple of ln2/32), on tiny |x| and on
    [-700, 700]; the CUDA library's exp is held to the same bound on the same inputs."""
    import torch
    g = np.random.default_rng(61)
    ln2_32 = np.log(2.0) / 32
    k = np.arange(-600, 40)
    x = np.concatenate([g.uniform(-20.0, 1.0, 400_000),
                        (k + 0.5) * ln2_32, (k + 0.5) * ln2_32 * (1 + 1e-15),
                        k * ln2_32, k * ln2_32 * (1 - 1e-15),
                        np.array([0.0, -0.0, 1e-300, -1e-20, 1e-12, -1e-8]),
                        g.uniform(-700.0, 700.0, 100_000)])
    mine, lib = pab.pab_exp_check(torch.as_tensor(x, device="cuda"))
    mine = mine.cpu().numpy()
    lib = lib.cpu().numpy()
    ref = np.exp(x.astype(np.longdouble))
    err_mine = np.abs((mine - ref) / ref).astype(np.float64)
    err_lib = np.abs((lib - ref) / ref).astype(np.float64)
    assert err_mine.max() <= 2.0 ** -51, (err_mine.max(), x[np.argmax(err_mine)])
    assert err_lib.max() <= 2.0 ** -51


def _ordered(v):
    """Doubles as integers in the order of their values (adjacent doubles one apart)."""
    b = np.asarray(v, dtype=np.float64).view(np.int64)
    return np.where(b < 0, -(b & 0x7FFFFFFFFFFFFFFF), b)


@pytest.mark.gpu
def test_integer_pipe_products_within_one_ulp():
    """Products and reciprocals formed from the significands with integer multiplies (the
    conservative-to-primitive pass, the FP64 trial's right-hand side): x y against the IEEE
    product, x^3 and 1/x against the correctly rounded exact values (exact rational arithmetic)
    are within 1 ulp everywhere and equal to them in all but a few per mille of draws (those
    within 2^-8 ulp of a tie); zero, signed, subnormal, infinite and NaN operands and results
    that overflow or underflow give the FP64 result."""
    import torch
    from fractions import Fraction
    g = np.random.default_rng(67)
    n = 200_000
    x = g.choice([-1.0, 1.0], n) * g.uniform(1.0, 2.0, n) * np.exp2(g.integers(-1060, 1060, n))
    y = g.choice([-1.0, 1.0], n) * g.uniform(1.0, 2.0, n) * np.exp2(g.integers(-1060, 1060, n))
    y[: n // 4] = 1.0 / g.uniform(1e8, 1e16, n // 4)  # 1/n_b of the pass
    x[: n // 4] = g.uniform(1e2, 1e10, n // 4) * g.choice([-1.0, 1.0], n // 4)
    top = np.nextafter(2.0, 0.0)  # all-ones significand: the rounding carries into the exponent
    special = np.array([0.0, -0.0, 5e-324, -1e-310, 2.0 ** -1022, np.inf, -np.inf, np.nan,
                        np.finfo(np.float64).max, 1.0, top, -top, 2.0 ** 341, 2.0 ** -342])
    xs, ys = np.meshgrid(special, special)
    x = np.concatenate([x, xs.ravel(), [top] * 4])
    y = np.concatenate([y, ys.ravel(), [top, np.nextafter(1.0, 2.0), 1.5, 2.0 ** -1000]])
    prod, cube, rcp = pab.pab_intmul_check(torch.as_tensor(x, device="cuda"),
                                           torch.as_tensor(y, device="cuda"))
    prod, cube, rcp = prod.cpu().numpy(), cube.cpu().numpy(), rcp.cpu().numpy()

    with np.errstate(all="ignore"):
        ref = x * y
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(prod), nan)
    d = np.abs(_ordered(prod[~nan]) - _ordered(ref[~nan]))
    assert d.max() <= 1, (d.max(), x[~nan][np.argmax(d)], y[~nan][np.argmax(d)])
    assert np.mean(d == 0) >= 0.99
    zero = ref == 0
    assert np.array_equal(np.signbit(prod[zero]), np.signbit(ref[zero]))

    finite = np.isfinite(x) & (x != 0)
    inrange = finite & (np.abs(x) > 2.0 ** -340) & (np.abs(x) < 2.0 ** 340)
    idx = np.flatnonzero(inrange)[:40_000]
    exact = np.array([float(Fraction(float(v)) ** 3) for v in x[idx]])
    dc = np.abs(_ordered(cube[idx]) - _ordered(exact))
    assert dc.max() <= 1, (dc.max(), x[idx][np.argmax(dc)])
    assert np.mean(dc == 0) >= 0.97
    rest = ~inrange
    with np.errstate(all="ignore"):
        ref3 = x[rest] * x[rest] * x[rest]
    nan3 = np.isnan(ref3)
    assert np.array_equal(np.isnan(cube[rest]), nan3)
    assert np.abs(_ordered(cube[rest][~nan3]) - _ordered(ref3[~nan3])).max() <= 2

    # 1/x against the correctly rounded exact reciprocal where x and 1/x are normal, against the
    # IEEE division elsewhere (zero, subnormal, infinite, NaN, and 1/x subnormal)
    normal = finite & (np.abs(x) >= 2.0 ** -1022) & (np.abs(x) < 2.0 ** 1022)
    idx = np.flatnonzero(normal)[:40_000]
    exact = np.array([float(1 / Fraction(float(v))) for v in x[idx]])
    dr = np.abs(_ordered(rcp[idx]) - _ordered(exact))
    assert dr.max() <= 1, (dr.max(), x[idx][np.argmax(dr)])
    assert np.mean(dr == 0) >= 0.99
    with np.errstate(all="ignore"):
        refr = 1.0 / x[~normal]
    nanr = np.isnan(refr)
    assert np.array_equal(np.isnan(rcp[~normal]), nanr)
    assert np.abs(_ordered(rcp[~normal][~nanr]) - _ordered(refr[~nanr])).max() <= 1
