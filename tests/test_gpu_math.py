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
