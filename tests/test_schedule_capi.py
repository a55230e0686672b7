"""The library's host-side schedule code (2MN arrays and the generalised multi-scale merge
of App. B) against the paper's printed example and the oracle's merge.  No GPU needed."""
import json
import os

import numpy as np
import pytest

from oracle.integrator import LAMBDA_2MN, leapfrog, merge, two_mn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def capi():
    from paper_1609_02652_gb300 import build, capi

    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return capi


def test_2mn_arrays(capi):
    for n, tau in [(1, 1.0), (3, 0.5), (8, 0.5)]:
        T, S = capi.pfmp_schedule_2mn(n, tau, LAMBDA_2MN)
        To, So = two_mn(n, tau)
        assert np.allclose(T, To, atol=1e-15) and np.allclose(S, So, atol=1e-15)
        assert abs(S.sum() - tau) < 1e-14 and abs(T.sum() - tau) < 1e-14


def test_merge_worked_example(capi):
    g = json.load(open(os.path.join(GOLDEN, "integrator_arrays.json")))["merged_demo"]
    lam = LAMBDA_2MN
    val = lambda x: x[0] + x[1] * lam
    T, S = capi.pfmp_schedule_merge([leapfrog(3, 1.0), two_mn(1, 1.0)])
    assert np.allclose(T, [val(x) for x in g["T"]], atol=1e-14)
    assert np.allclose(S[0], [val(x) for x in g["S1"]], atol=1e-14)
    assert np.allclose(S[1], [val(x) for x in g["S2"]], atol=1e-14)


@pytest.mark.parametrize("steps", [(8, 16), (4, 10, 25), (4, 10, 24, 60)])
def test_merge_matches_oracle(capi, steps):
    schemes = [two_mn(n, 1.0) for n in steps]
    T, S = capi.pfmp_schedule_merge(schemes)
    To, So = merge(schemes)
    assert len(T) == len(To)
    assert np.allclose(T, To, atol=1e-13) and np.allclose(S, np.array(So), atol=1e-13)


def test_merge_rejects_bad_input(capi):
    with pytest.raises(capi.PfmpError):
        capi.pfmp_schedule_merge([two_mn(8, 1.0)], cap=3)
