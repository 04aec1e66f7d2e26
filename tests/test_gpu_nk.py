"""Newton-Krylov-hookstep on the pipe flow (batched guesses).  The Newton
residual certifies an invariant solution; it is re-checked here with the
oracle's own time stepper (independent of the GPU path)."""
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


def test_nk_finds_equilibrium_and_oracle_certifies_it(opf):
    N, K, M, m_p, alpha, Re = 12, 3, 3, 1, 1.25, 100.0
    lam = inputs.laminar_state(N, K, M)
    guesses = [lam + inputs.seeded_state(N, K, M, m_p, alpha, a, 31 + i, laminar=False)
               for i, a in enumerate((1e-3, 3e-2))]
    T0 = 0.5
    states, T, s, res, it = opf.opf_nk_solve(N, K, M, m_p, alpha, Re, guesses, [T0, T0], [0.0, 0.0],
                                             fix_T=1, fix_s=1, dt=0.05, tol=1e-11, max_krylov=40,
                                             gmres_tol=1e-4, max_newton=20)
    assert (res < 1e-11).all(), res
    assert (it >= 1).all()
    o = Oracle(Params(N, K, M, m_p, alpha, Re, T0 / 10))
    for u in states:
        # the only invariant solution near these guesses at Re = 100 is laminar flow
        assert np.abs(u - lam).max() < 1e-9
        v = o.step(u, 10)
        assert np.linalg.norm(v - u) / np.linalg.norm(u) < 1e-10


def test_nk_free_period_and_shift_rejects_nothing_silently(opf):
    """With T and s free the phase conditions enter the system; on a state
    with axial structure the solver still reduces the residual and keeps the
    unknowns finite."""
    N, K, M, m_p, alpha, Re = 12, 3, 3, 1, 1.25, 100.0
    lam = inputs.laminar_state(N, K, M)
    g = lam + inputs.seeded_state(N, K, M, m_p, alpha, 1e-2, 7, laminar=False)
    u0 = g.copy()
    states, T, s, res, it = opf.opf_nk_solve(N, K, M, m_p, alpha, Re, [g], [0.5], [0.1],
                                             dt=0.05, tol=1e-9, max_krylov=40, gmres_tol=1e-4,
                                             max_newton=6)
    h = opf.opf_create(N, K, M, m_p, alpha, Re, 0.05)
    opf.opf_set_state(h, u0)
    opf.opf_step(h, 10)
    r0 = np.linalg.norm(opf.opf_get_state(h) - u0) / np.linalg.norm(u0)
    assert np.isfinite(T).all() and np.isfinite(s).all()
    assert res[0] < 0.5 * r0


def test_multiple_shooting_finds_equilibrium_and_oracle_certifies_it(opf):
    """Two sections per orbit: the sections converge to the same invariant
    solution (laminar flow at Re = 100) and the oracle certifies it.  With
    half-period sections of an equilibrium the Jacobian's small eigenvalues
    halve, so GMRES needs more iterations and Newton more steps than single
    shooting."""
    N, K, M, m_p, alpha, Re = 12, 3, 3, 1, 1.25, 100.0
    lam = inputs.laminar_state(N, K, M)
    guesses = [[lam + inputs.seeded_state(N, K, M, m_p, alpha, a, 51 + 2 * i + q, laminar=False) for q in range(2)]
               for i, a in enumerate((1e-3, 2e-2))]
    T0 = 0.5
    secs, T, s, res, it = opf.opf_nk_solve_ms(N, K, M, m_p, alpha, Re, guesses, [T0, T0], [0.0, 0.0],
                                              fix_T=1, fix_s=1, dt=0.05, tol=1e-11, max_krylov=40,
                                              gmres_tol=1e-4, max_newton=50)
    assert (res < 1e-11).all(), res
    o = Oracle(Params(N, K, M, m_p, alpha, Re, T0 / 10))
    for sec in secs:
        for u in sec:
            assert np.abs(u - lam).max() < 1e-9
            assert np.linalg.norm(o.step(u, 5) - u) / np.linalg.norm(u) < 1e-10


def test_multiple_shooting_with_one_section_equals_single_shooting(opf):
    N, K, M, m_p, alpha, Re = 12, 3, 3, 1, 1.25, 100.0
    lam = inputs.laminar_state(N, K, M)
    g = lam + inputs.seeded_state(N, K, M, m_p, alpha, 1e-2, 61, laminar=False)
    kw = dict(dt=0.05, tol=1e-9, max_krylov=30, gmres_tol=1e-4, max_newton=4)
    a = opf.opf_nk_solve(N, K, M, m_p, alpha, Re, [g], [0.5], [0.1], **kw)
    b = opf.opf_nk_solve_ms(N, K, M, m_p, alpha, Re, [[g]], [0.5], [0.1], **kw)
    assert abs(a[3][0] - b[3][0]) <= 1e-9 * max(a[3][0], 1e-300) + 1e-14
    np.testing.assert_allclose(b[0][0][0], a[0][0], rtol=0, atol=1e-12)
