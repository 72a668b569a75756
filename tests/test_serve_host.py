"""Host-side checks of the serving entry points (no GPU needed): option
validation, rejection of a request whose estimated footprint exceeds the
budget, and unknown request ids."""
from __future__ import annotations

import pytest

import paper_2306_05789_gb300 as rt
import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_05789_gb300 import build
    build.build()


def test_invalid_server_options_are_rejected():
    for kw in ({"hbm_budget": 0}, {"slots": 0}, {"slots": 65}, {"max_bypass": -1}, {"tol": -1.0}):
        with pytest.raises(rt.RtError) as e:
            rt.Server(rt.hparams(), **kw)
        assert e.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError):
        rt.Server(rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))


def test_request_larger_than_the_budget_is_refused_at_submit():
    srv = rt.Server(rt.hparams(), hbm_budget=1000, slots=1)
    p = W.cube_problem(8, W.sinprod_kappa(0.5), W.midpoint_freqs(2), R0=0.5)
    with pytest.raises(rt.RtError) as e:
        srv.submit(p)
    assert e.value.code == rt.RT_ENOMEM
    assert srv.info()["submitted"] == 0
    srv.free()


def test_malformed_request_and_unknown_id_are_rejected():
    srv = rt.Server(rt.hparams(), hbm_budget=10**9, slots=1)
    p = W.cube_problem(6, W.sinprod_kappa(0.5), W.midpoint_freqs(1), R0=0.5)
    p.tet[0, 0] = p.N + 5
    with pytest.raises(rt.RtError) as e:
        srv.submit(p)
    assert e.value.code == rt.RT_EINVAL
    srv._dims[12345] = (1, 8)
    with pytest.raises(rt.RtError) as e:
        srv.poll(12345)
    assert e.value.code == rt.RT_EINVAL
    srv.free()
