"""The library's step balancing and cost function (host logic, no GPU) against the
oracle's (Sec. 2.4 eq. force_tune; Sec. 3.1 eqs. cost_func, error_corrected)."""
import numpy as np
import pytest

from oracle.tuning import balance_steps, cost


def test_balance_steps_matches_oracle():
    from paper_1609_02652_gb300 import capi

    rng = np.random.default_rng(5)
    for _ in range(50):
        f = list(rng.uniform(0.05, 20.0, size=rng.integers(1, 6)))
        n0 = int(rng.integers(1, 12))
        assert capi.pfmp_balance_steps(f, n0) == balance_steps(f, n0)
    with pytest.raises(capi.PfmpError):
        capi.pfmp_balance_steps([1.0, 0.0], 4)


def test_cost_matches_oracle():
    from paper_1609_02652_gb300 import capi

    rng = np.random.default_rng(6)
    for n in (2, 5, 40):
        acc = list(rng.integers(0, 2, size=n))
        acc[0] = 1
        nmat = list(rng.uniform(500, 900, size=n))
        dh = list(rng.normal(0.1, 0.4, size=n))
        got = capi.pfmp_cost(acc, nmat, dh, 12.5)
        ref = cost(acc, nmat, dh, 12.5)
        for k, v in ref.items():
            assert abs(getattr(got, k) - v) <= 1e-12 * max(1.0, abs(v)), k
    with pytest.raises(capi.PfmpError):
        capi.pfmp_cost([1], [1.0], [0.0])
