"""Row a1 (the bin table, Sec. 2.2) of the library against the oracle, on the CPU.

pab_bin_table returns the table and default n_b a handle of the same config holds (the
library builds both on the host), so this parity needs no GPU.  The two sides compute the
nodes and the normalised Simpson weights in independent FP64 code, so they agree to a few
ulp (4e-15 relative; the nodes agree bit for bit, the weights within 2 ulp); the default n_b must give the configured void fraction at equilibrium
through the oracle's own moments (Eq. e:ndf)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2511_21031_gb300 import pab, workloads

RTOL = 4e-15  # a few ulp of FP64: a normalising sum taken in a different order


@pytest.mark.parametrize("B", [1, 3, 11, 21, 31, 51, 63])
@pytest.mark.parametrize("s", [0.2, 0.3, 0.5, 0.7])
def test_lognormal_table_and_default_nb_match_the_oracle(B, s):
    R0ref, K, alpha0 = 10e-6, 5.0, 4e-5
    R0, w, nb = pab.pab_bin_table(n_cells=1, n_bins=B, R0ref=R0ref, s_lognormal=s, span_K=K,
                                  alpha0=alpha0)
    oR0, ow = oracle.bins(B, R0ref, s, K)
    np.testing.assert_allclose(R0, oR0, rtol=RTOL, atol=0.0)
    np.testing.assert_allclose(w, ow, rtol=RTOL, atol=1e-300)
    assert nb == pytest.approx(oracle.equilibrium_nb(alpha0, oR0, ow), rel=RTOL)
    P = oracle.Params(**workloads.WATER)
    Req = np.asarray(oR0, dtype=np.float64).reshape(B, 1)
    m = oracle.moments(P, oR0, ow, np.array([nb]), Req, np.zeros_like(Req))
    assert m[1, 0] == pytest.approx(alpha0, rel=RTOL)


def test_explicit_table_is_taken_as_given():
    R0 = (ctypes.c_double * 3)(5e-6, 1e-5, 2e-5)
    w = (ctypes.c_double * 3)(0.25, 0.5, 0.25)
    dp = ctypes.POINTER(ctypes.c_double)
    got_R0, got_w, nb = pab.pab_bin_table(n_cells=1, n_bins=3, R0_host=ctypes.cast(R0, dp),
                                          w_host=ctypes.cast(w, dp), alpha0=1e-3)
    assert got_R0 == list(R0) and got_w == list(w)
    assert nb == pytest.approx(oracle.equilibrium_nb(1e-3, list(R0), list(w)), rel=RTOL)


@pytest.mark.parametrize("bad", [dict(n_bins=4), dict(n_bins=21, s_lognormal=0.0),
                                 dict(n_bins=21, span_K=-1.0), dict(n_cells=0), dict(R0ref=0.0)])
def test_tables_pab_create_refuses_are_refused(bad):
    with pytest.raises(pab.PabError):
        pab.pab_bin_table(**{"n_cells": 1, **bad})
