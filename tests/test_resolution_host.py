"""Resolution change of states (host): the oracle's interpolation is exact on
parity-consistent polynomials, the library equals the oracle, equal sizes are
the identity, Fourier truncation / zero padding are exact, and a smooth state
survives a fine -> coarse -> fine round trip."""
import numpy as np
import pytest

from oracle.opf_oracle import change_resolution, mesh
from paper_1705_03838_gb300 import inputs


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def poly_state(N, K, M, m_p, seed):
    """Each (c, m, k) profile a polynomial of degree <= 8 with the field's axis
    parity: r^p (a0 + a1 r^2 + ...), p = 0 or 1."""
    rng = np.random.default_rng(seed)
    r = mesh(N)
    U = np.zeros((3, M, 2 * K - 1, N), dtype=np.complex128)
    for c in range(3):
        for m in range(M):
            mt = m_p * m
            p = mt % 2 if c == 2 else (mt + 1) % 2
            for kk in range(2 * K - 1):
                a = rng.normal(size=4) + 1j * rng.normal(size=4)
                U[c, m, kk] = r ** p * sum(a[q] * r ** (2 * q) for q in range(4))
    return U


def test_oracle_interpolation_exact_on_polynomials():
    U = poly_state(20, 3, 3, 2, 1)
    V = change_resolution(U, 33, 3, 3, 2)
    np.testing.assert_allclose(V, poly_state(33, 3, 3, 2, 1), rtol=0, atol=1e-11)


def test_library_equals_oracle(opf):
    U = inputs.seeded_state(24, 5, 4, 1, 1.25, 0.1, 3)
    for (N2, K2, M2) in ((24, 5, 4), (31, 3, 6), (16, 7, 2)):
        a = opf.opf_change_resolution(U, N2, K2, M2, 1)
        b = change_resolution(U, N2, K2, M2, 1)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_identity_and_fourier_truncation(opf):
    U = inputs.seeded_state(24, 5, 4, 2, 1.25, 0.1, 4)
    np.testing.assert_array_equal(opf.opf_change_resolution(U, 24, 5, 4, 2), U)
    V = opf.opf_change_resolution(U, 24, 3, 2, 2)
    np.testing.assert_array_equal(V, U[:, :2, 2:7])
    W = opf.opf_change_resolution(V, 24, 5, 4, 2)
    assert np.abs(W[:, 2:]).max() == 0 and np.abs(W[:, :, :2]).max() == 0 and np.abs(W[:, :, 7:]).max() == 0
    np.testing.assert_array_equal(W[:, :2, 2:7], V)


def test_round_trip_of_a_smooth_state(opf):
    U = inputs.seeded_state(48, 6, 6, 1, 1.25, 0.1, 5)
    V = opf.opf_change_resolution(opf.opf_change_resolution(U, 64, 6, 6, 1), 48, 6, 6, 1)
    assert np.linalg.norm(V - U) / np.linalg.norm(U) < 1e-6


def test_rejects_bad_sizes(opf):
    U = inputs.seeded_state(8, 2, 2, 1, 1.25, 0.1, 6)
    with pytest.raises(opf.OpfError):
        opf.opf_change_resolution(U, 16, 2, 2, 1)  # source N < 9
