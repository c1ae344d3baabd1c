"""The gas-term node table the library builds on the host, checked on the CPU.

A handle evaluates the polytropic gas factor (R0/R)^(3 gamma) = x^(-3 gamma), x = R/R0, as the
binomial series around the nearest node x_j = q^j of this table (pab_gas_table returns the table
and its bound exactly as a handle builds them).  Checked here against the mathematics, not
against the library's formulas:
- the nodes are geometric, centred on x = 1, and cover x in [1/25, 25];
- the centre node holds the binomial coefficients C(-3 gamma, k);
- the nearest node of any x in log x, and either node at a geometric mid-point, lies within
  the stated bound dmax;
- there the series, summed exactly from the stored FP64 values, equals x^(-3 gamma) from
  50-digit decimal arithmetic to within a few ulp over the whole range (truncation below half
  an ulp plus the rounding of the stored coefficients), for gamma = 1, 1.4 and 5/3."""
import decimal
import math

import numpy as np
import pytest

from paper_2511_21031_gb300 import pab

ULP = 2.0 ** -52
TOL = 3 * ULP  # half an ulp of truncation plus the roundings of the stored node and coefficients


def _exact_pow(x: float, a: float) -> decimal.Decimal:
    with decimal.localcontext() as ctx:
        ctx.prec = 50
        return decimal.Decimal(x) ** decimal.Decimal(-a)


def _series(node, x: float) -> decimal.Decimal:
    with decimal.localcontext() as ctx:
        ctx.prec = 50
        d = decimal.Decimal(x) - decimal.Decimal(float(node[0]))
        return sum(decimal.Decimal(float(c)) * d ** k for k, c in enumerate(node[1:]))


@pytest.mark.parametrize("gamma", [1.0, 1.4, 5.0 / 3.0])
def test_nodes_are_geometric_and_cover_the_range(gamma):
    tab, dmax = pab.pab_gas_table(gamma)
    x = tab[:, 0]
    n = x.shape[0]
    assert n % 2 == 1 and x[n // 2] == 1.0
    q = x[n // 2 + 1]
    assert np.allclose(x[1:] / x[:-1], q, rtol=1e-13, atol=0.0)
    assert x[0] <= 1.0 / 25.0 and x[-1] >= 25.0
    assert math.sqrt(q) - 1.0 <= dmax          # the nearest node is always within the bound
    a = 3.0 * gamma
    c = 1.0
    for k in range(1, tab.shape[1]):
        if k - 1 < 4:
            assert tab[n // 2, k] == pytest.approx(c, rel=4 * ULP)
            c *= (-a - (k - 1)) / k
        else:
            assert tab[n // 2, k] == 0.0


@pytest.mark.parametrize("gamma", [1.0, 1.4, 5.0 / 3.0])
def test_series_at_the_nearest_node_is_the_gas_factor(gamma):
    tab, dmax = pab.pab_gas_table(gamma)
    a = 3.0 * gamma
    n = tab.shape[0]
    J = n // 2
    lq = math.log(tab[J + 1, 0])
    g = np.random.Generator(np.random.PCG64(11))
    xs = np.exp(g.uniform(math.log(1.0 / 25.0), math.log(25.0), size=1500))
    worst = 0.0
    for x in xs:
        j = int(round(math.log(x) / lq))
        node = tab[j + J]
        assert abs(x / node[0] - 1.0) <= dmax
        ex = _exact_pow(float(x), a)
        worst = max(worst, abs(float((_series(node, float(x)) - ex) / ex)))
    # geometric mid-points between nodes, where a rounded index may pick either neighbour
    for j in range(-J, J, max(1, n // 400)):
        lo, hi = tab[j + J], tab[j + J + 1]
        x = math.sqrt(lo[0] * hi[0])
        ex = _exact_pow(x, a)
        for node in (lo, hi):
            assert abs(x / node[0] - 1.0) <= dmax
            worst = max(worst, abs(float((_series(node, x) - ex) / ex)))
    assert worst <= TOL, worst


def test_invalid_gamma_is_refused():
    for bad in (0.0, -1.4, float("nan"), float("inf")):
        with pytest.raises(pab.PabError):
            pab.pab_gas_table(bad)
