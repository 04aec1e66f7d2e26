"""Newton-Krylov-hookstep core (native, CPU) on synthetic problems whose
solutions are known: a linear system (GMRES exact), a coupled nonlinear
system, a problem where the plain Newton step diverges (trust region needed),
and several problems solved in lockstep."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def fd_jv(F):
    def JV(idx, xs, vs):
        out = []
        for i, x, v in zip(idx, xs, vs):
            eps = 1e-7 * max(1.0, np.linalg.norm(x)) / max(np.linalg.norm(v), 1e-300)
            out.append((F([i], [x + eps * v])[0] - F([i], [x])[0]) / eps)
        return out
    return JV


def test_linear_system_solved_by_gmres(opf):
    rng = np.random.default_rng(1)
    n = 30
    A = np.eye(n) * 4 + rng.normal(size=(n, n)) * 0.3
    b = rng.normal(size=n)
    F = lambda idx, xs: [A @ x - b for x in xs]
    JV = lambda idx, xs, vs: [A @ v for v in vs]
    x, res, it = opf.opf_nk_core(np.zeros((1, n)), F, JV, tol=1e-12, gmres_tol=1e-14, max_krylov=n + 1,
                                 delta0=1e3)
    assert np.linalg.norm(x[0] - np.linalg.solve(A, b)) < 1e-10
    assert res[0] < 1e-12 and it[0] <= 2


def test_nonlinear_system(opf):
    n = 12
    c = np.linspace(0.5, 3.0, n)

    def F(idx, xs):
        out = []
        for x in xs:
            f = x ** 3 + 2 * x - c
            f[:-1] += 0.1 * x[1:] ** 2
            out.append(f)
        return out

    x, res, it = opf.opf_nk_core(np.zeros((1, n)), F, fd_jv(F), tol=1e-12, gmres_tol=1e-10,
                                 max_krylov=n + 1, delta0=1.0)
    assert res[0] < 1e-11
    assert np.abs(F([0], [x[0]])[0]).max() < 1e-11


def test_trust_region_rescues_diverging_newton(opf):
    """Newton on atan(x) = 0 diverges from |x0| > 1.39; the hookstep does not."""
    F = lambda idx, xs: [np.arctan(x) for x in xs]
    JV = lambda idx, xs, vs: [v / (1 + x ** 2) for x, v in zip(xs, vs)]
    x, res, it = opf.opf_nk_core(np.array([[3.0]]), F, JV, tol=1e-13, gmres_tol=1e-12, max_krylov=2,
                                 delta0=0.5, max_newton=60)
    assert abs(x[0, 0]) < 1e-12 and res[0] < 1e-13
    # the plain Newton iteration from the same start blows up
    y = 3.0
    for _ in range(5):
        y = y - np.arctan(y) * (1 + y * y)
    assert abs(y) > 100


def test_problems_in_lockstep(opf):
    cs = [1.0, 2.0, 5.0]
    calls = []

    def F(idx, xs):
        calls.append(list(idx))
        return [x ** 2 - cs[i] for i, x in zip(idx, xs)]

    JV = lambda idx, xs, vs: [2 * x * v for x, v in zip(xs, vs)]
    x0 = np.ones((3, 1)) * 3.0
    x, res, it = opf.opf_nk_core(x0, F, JV, tol=1e-13, gmres_tol=1e-12, max_krylov=2, delta0=10.0)
    assert np.allclose(x[:, 0], np.sqrt(cs), rtol=0, atol=1e-12)
    assert any(len(c) > 1 for c in calls)  # batched evaluations
