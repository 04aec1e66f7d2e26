"""Leading eigenvalues by Arnoldi: the oracle and the library's host core
against operators with a spectrum known by construction, the library's
Hessenberg QR against a companion matrix of known roots, and the oracle's
Floquet multipliers of an axisymmetric swirl against the closed form
exp(-j_{1,n}^2 T / Re)."""
import numpy as np
import pytest
from scipy.special import jn_zeros

from oracle import floquet_oracle as fo
from oracle.opf_oracle import Oracle, Params
from paper_1705_03838_gb300 import inputs


def known_operator(n, seed):
    """A = Q D Q^T with D holding real eigenvalues and 2 x 2 rotation blocks."""
    rng = np.random.default_rng(seed)
    lam = [0.95, 0.9 * np.exp(0.3j), 0.8, 0.7 * np.exp(-1.1j), 0.5]
    D = np.zeros((n, n))
    i = 0
    exact = []
    for l in lam:
        if np.imag(l) == 0:
            D[i, i] = np.real(l)
            exact.append(np.real(l))
            i += 1
        else:
            r, t = abs(l), np.angle(l)
            D[i:i + 2, i:i + 2] = r * np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
            exact += [l, np.conj(l)]
            i += 2
    D[np.arange(i, n), np.arange(i, n)] = 0.3 * rng.uniform(-1, 1, n - i)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return Q @ D @ Q.T, np.array(exact)


def close_sets(a, b, tol):
    a, b = list(a), list(b)
    for x in a:
        j = int(np.argmin([abs(x - y) for y in b]))
        if abs(x - b[j]) > tol:
            return False
        b.pop(j)
    return True


def test_oracle_arnoldi_on_known_spectrum():
    A, exact = known_operator(150, 1)
    ev = fo.arnoldi(lambda v: A @ v, np.random.default_rng(2).normal(size=150), 60)
    assert close_sets(ev[:len(exact)], exact, 1e-10)


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def test_library_arnoldi_on_known_spectrum(opf):
    A, exact = known_operator(200, 3)
    B, exact_b = known_operator(200, 4)
    v0 = np.random.default_rng(5).normal(size=(2, 200))
    ev, res, k = opf.opf_arnoldi_core(v0, lambda idx, vs: [(A if i == 0 else B) @ v for i, v in zip(idx, vs)],
                                      60, 7)
    assert close_sets(ev[0][:7], exact, 1e-12) and close_sets(ev[1][:7], exact_b, 1e-12)
    assert (res < 1e-10).all() and (k == 60).all()


def test_library_arnoldi_stops_on_invariant_subspace(opf):
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.normal(size=(50, 3)))
    A = Q @ np.diag([2.0, -1.0, 0.5]) @ Q.T  # rank 3
    ev, res, k = opf.opf_arnoldi_core(rng.normal(size=(1, 50)), lambda idx, vs: [A @ v for v in vs], 20, 3)
    assert k[0] <= 4
    assert close_sets(ev[0], [2.0, -1.0, 0.5], 1e-12)


def test_library_hessenberg_qr_on_companion_matrix(opf):
    """A companion matrix is upper Hessenberg after a permutation; its
    eigenvalues are the polynomial's roots (repeated and complex ones)."""
    roots = np.array([1.5, 1.5, -0.5, 0.2 + 0.9j, 0.2 - 0.9j, -1.1 + 0.3j, -1.1 - 0.3j])
    c = np.poly(roots).real
    n = len(roots)
    C = np.zeros((n, n))
    C[0, :] = -c[1:]
    C[np.arange(1, n), np.arange(n - 1)] = 1.0
    ev, res, k = opf.opf_arnoldi_core(np.ones((1, n)), lambda idx, vs: [C @ v for v in vs], n, n)
    assert close_sets(ev[0], roots, 2e-6)  # a double root is sensitive at sqrt(machine epsilon)


def test_oracle_floquet_of_axisymmetric_swirl():
    """u_theta(r) perturbations of Hagen-Poiseuille with k = m = 0 decay
    independently: multipliers exp(-j_{1,n}^2 T / Re) (plus time and radial
    discretisation errors, ~1e-5 here).  The finite-difference products carry
    round-off into the other modes, so the swirl multipliers are looked up
    among the Ritz values rather than expected to lead."""
    N, K, M, Re, T, dt = 32, 2, 2, 100.0, 1.0, 0.01
    o = Oracle(Params(N, K, M, 1, 1.25, Re, dt))
    U = inputs.laminar_state(N, K, M)
    start = np.zeros_like(U)
    start[1, 0, K - 1] = np.random.default_rng(7).normal(size=N)
    start[1, 0, K - 1, -1] = 0.0
    ev = fo.floquet(o, U, T, 0.0, fo.pack(start, K, M), 10)
    for mu in np.exp(-jn_zeros(1, 3) ** 2 * T / Re):
        assert np.min(np.abs(ev - mu)) < 2e-5 * mu, (mu, ev)
