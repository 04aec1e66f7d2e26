"""Mixed precision (FP32 transforms and u' x w', FP64 solves, boundary
correction and base-flow terms) against the FP64 oracle.

Target: relative energy error <= 1e-5 over 100 steps of the small workload;
the relative L2 error of all coefficients is held well below FP32 rounding of
the perturbation."""
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


@pytest.mark.parametrize("N,K,M,m_p,amp", [(16, 4, 6, 1, 0.1), (12, 3, 4, 2, 0.3), (32, 16, 16, 1, 0.01)])
def test_mixed_nonlinear_term(opf, N, K, M, m_p, amp):
    alpha, Re = 1.25, 1000.0
    U0 = inputs.seeded_state(N, K, M, m_p, alpha, amp, 31)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.01)
    opf.opf_set_option(h, "precision", 1)
    got = opf.opf_nonlinear(h, U0)
    o = Oracle(Params(N, K, M, m_p, alpha, Re, 0.01))
    want = o.nonlinear(U0)
    # FP32 only touches u' x w', whose size is ~amp^2; the rest is FP64
    pert = want - o.nonlinear(inputs.laminar_state(N, K, M))
    err = np.abs(got - want).max()
    assert err <= 2e-6 * max(np.abs(pert).max(), 1e-300) + 1e-13 * np.abs(want).max()


def test_mixed_small_workload_100_steps(opf):
    w = inputs.WORKLOADS["small"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    o = Oracle(Params(*args))
    U0 = inputs.workload_state("small")
    ref = o.step(U0, 100)
    h = opf.opf_create(*args)
    opf.opf_set_option(h, "precision", 1)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 100)
    U = opf.opf_get_state(h)
    e, e_ref = opf.opf_energy(h), o.energy(ref)
    rel_energy = abs(e[0] - e_ref[0]) / e_ref[0]
    lam = inputs.laminar_state(w["N"], w["K"], w["M"])
    rel_pert = np.linalg.norm(U - ref) / np.linalg.norm(ref - lam)
    print(f"mixed small 100 steps: rel energy err {rel_energy:.3e}, perturbation-relative L2 {rel_pert:.3e}")
    assert rel_energy <= 1e-5
    assert rel_pert <= 1e-4


def test_mixed_medium_workload_few_steps(opf):
    w = inputs.WORKLOADS["medium"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    o = Oracle(Params(*args))
    U0 = inputs.workload_state("medium")
    ref = o.step(U0, 3)
    h = opf.opf_create(*args)
    opf.opf_set_option(h, "precision", 1)
    opf.opf_set_state(h, U0)
    opf.opf_step(h, 3)
    U = opf.opf_get_state(h)
    lam = inputs.laminar_state(w["N"], w["K"], w["M"])
    rel_pert = np.linalg.norm(U - ref) / np.linalg.norm(ref - lam)
    rel_energy = abs(opf.opf_energy(h)[0] - o.energy(ref)[0]) / o.energy(ref)[0]
    print(f"mixed medium 3 steps: rel energy err {rel_energy:.3e}, perturbation-relative L2 {rel_pert:.3e}")
    assert rel_energy <= 1e-6 and rel_pert <= 1e-5
