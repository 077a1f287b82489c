"""Host-side checks of the serving form (no GPU): the server's argument
checks and the seeded Poisson workload."""
import numpy as np
import pytest

import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth


def test_server_create_refuses_bad_options():
    W = synth.make_weights(lic.HYPERPRIOR, 32, 48)
    for kw in (dict(max_batch=0), dict(max_batch=65), dict(lanes=0), dict(lanes=9), dict(max_pending=0),
               dict(max_wait_ms=-1.0), dict(hbm_budget=0)):
        with pytest.raises(lic.LicError) as e:
            lic.Server(lic.HYPERPRIOR, 32, 48, W, **kw)
        assert e.value.code == lic.E_INVALID_ARG, kw
    with pytest.raises(lic.LicError):
        lic.Server(5, 32, 48, W)


def test_poisson_arrivals_rate_and_gaps():
    """Each of the 16 streams is a Poisson process of 30 frames/s: over 20 s
    its count is 600 +- 5 sqrt(600), its gaps average 1/30 s and their
    standard deviation equals their mean (exponential)."""
    arr = synth.poisson_arrivals(20.0)
    assert [a[0] for a in arr] == sorted(a[0] for a in arr)
    assert all(0.0 <= a[0] < 20.0 for a in arr)
    res = {a[1]: (a[2], a[3]) for a in arr}
    assert sorted(set(res.values())) == [(480, 640), (720, 1280), (1080, 1920)]
    assert sum(1 for r in res.values() if r == (1080, 1920)) == 4
    for sid in range(16):
        t = np.array([a[0] for a in arr if a[1] == sid])
        assert abs(len(t) - 600) <= 5 * np.sqrt(600), sid
        g = np.diff(t)
        assert abs(g.mean() - 1 / 30) < 0.2 / 30
        assert abs(g.std() / g.mean() - 1.0) < 0.2
    assert synth.poisson_arrivals(1.0) == synth.poisson_arrivals(1.0)
