"""Automatic time-step control (paper section 2): the GPU picks dt from the
CFL condition; the oracle replays the same dt sequence and must agree."""
import numpy as np
import pytest

from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


@pytest.mark.parametrize("precision", [0, 1])
def test_cfl_dt_sequence_replayed_by_oracle(opf, precision):
    N, K, M, m_p, alpha, Re = 16, 4, 4, 1, 1.25, 500.0
    dt0, C = 0.05, 0.35
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, 0.3, 77)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, dt0)
    opf.opf_set_option(h, "precision", precision)
    opf.opf_set_option(h, "cfl", C)
    opf.opf_set_state(h, U0)
    dts = [dt0]
    for _ in range(8):
        opf.opf_step(h, 1)
        dts.append(opf.opf_get_dt(h))
    U = opf.opf_get_state(h)
    assert len(set(dts)) >= 2, "the CFL limit never changed dt"
    assert all(d <= dt0 * (1 + 1e-15) for d in dts)
    assert abs(opf.opf_get_time(h) - sum(dts[:-1])) < 1e-14
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt0))
    V = U0
    for d in dts[:-1]:
        if d != o.p.dt:
            o.p.dt = d
            o._lu.clear()
        V = o.step(V, 1)
    err = np.linalg.norm(U - V) / np.linalg.norm(V)
    assert err < (1e-12 if precision == 0 else 1e-7)


def test_cfl_number_bounded(opf):
    N, K, M, alpha = 24, 6, 6, 1.0
    h = opf.opf_create(N, K, M, 1, alpha, 1000.0, 0.02)
    opf.opf_set_option(h, "precision", 1)
    opf.opf_set_option(h, "cfl", 0.5)
    opf.opf_set_option(h, "dt_max", 0.02)
    opf.opf_set_state(h, inputs.seeded_state(N, K, M, 1, alpha, 0.3, 5))
    for _ in range(6):
        opf.opf_step(h, 1)
        # after the update, the step just taken used at most 10 % more than C
        assert opf.opf_get_option(h, "cfl_number") <= 0.5 * 1.1 + 1e-12
    assert opf.opf_get_dt(h) <= 0.02
