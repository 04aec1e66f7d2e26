"""CPU-only checks of the C ABI library: it loads, exports every symbol that
include/opf.h declares, validates arguments, and its host-side setup (mesh,
stencils, quadrature) agrees with the independently written oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.opf_oracle import fd_matrices, mesh, quadrature_weights
from paper_1705_03838_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def opf():
    from paper_1705_03838_gb300 import build, opf as _opf

    build.build()
    _opf.lib()
    return _opf


def declared_functions():
    text = open(os.path.join(ROOT, "include", "opf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(opf_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(opf):
    names = declared_functions()
    assert len(names) >= 18
    L = ctypes.CDLL(opf.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_setup_query_rejects_bad_arguments(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(8, 4, 4, 1, 1.25, 100.0, 0.01, "r")  # N < 9
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(16, 4, 4, 1, 1.25, 100.0, 0.01, "nonsense")


@pytest.mark.parametrize("N", [9, 16, 33])
def test_host_stencils_match_oracle(opf, N):
    r = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "r")
    assert np.abs(r - mesh(N)).max() < 1e-15
    wq = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "wq")
    assert np.abs(wq - quadrature_weights(mesh(N))).max() < 1e-15
    for what, idx in (("d1", 0), ("d2", 1)):
        w = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, what).reshape(2, N, 9)
        for par, sgn in ((0, 1), (1, -1)):
            ref = fd_matrices(mesh(N), sgn)[idx]
            A = np.zeros((N, N))
            for n in range(N):
                lo = min(max(n - 4, 0), N - 9)
                A[n, lo:lo + 9] = w[par, n]
            assert np.abs(A - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("N", [12, 24])
def test_host_setup_on_a_user_mesh_matches_oracle(opf, N):
    """A user radial mesh (opf_setup_query_mesh / opf_create_mesh): points,
    quadrature and both stencils against the oracle on the same points."""
    rm = inputs.stretched_mesh(N)
    r = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "r", r=rm)
    assert np.array_equal(r, rm)
    wq = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, "wq", r=rm)
    assert np.abs(wq - quadrature_weights(rm)).max() < 1e-15
    for what, idx in (("d1", 0), ("d2", 1)):
        w = opf.opf_setup_query(N, 4, 4, 1, 1.25, 100.0, 0.01, what, r=rm).reshape(2, N, 9)
        for par, sgn in ((0, 1), (1, -1)):
            ref = fd_matrices(rm, sgn)[idx]
            A = np.zeros((N, N))
            for n in range(N):
                lo = min(max(n - 4, 0), N - 9)
                A[n, lo:lo + 9] = w[par, n]
            assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


def test_user_mesh_is_validated(opf):
    rm = inputs.stretched_mesh(12)
    for bad in (rm[::-1], np.concatenate([rm[:-1], [0.99]]), np.concatenate([[0.0], rm[1:]]),
                np.concatenate([rm[:5], rm[4:5], rm[6:]])):
        with pytest.raises(opf.OpfError):
            opf.opf_setup_query(12, 4, 4, 1, 1.25, 100.0, 0.01, "r", r=bad)


def test_flux_response_is_positive_and_vanishes_at_wall(opf):
    G = opf.opf_setup_query(24, 4, 4, 1, 1.25, 2000.0, 0.01, "G")
    assert G[-1] == 0.0 and np.all(G[:-1] > 0)


def test_setup_rejects_unfactorable_sizes(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(4, 4, 4, 1, 1.25, 100.0, 0.01, "r")


def column_substitution(F, b):
    """The banded substitution in the order the solve kernel takes it: column
    by column, on one operator's factors in the device layout (13 N values:
    L(c+1+t, c), L(c+5+t, c) read in the last nine columns only, 1/U(c,c),
    U(c-1-t, c) / U(c-1-t, c-1-t))."""
    N = len(b)
    L, Lw = F[:4 * N].reshape(N, 4), F[4 * N:8 * N].reshape(N, 4)
    dg, Uc = F[8 * N:9 * N], F[9 * N:].reshape(N, 4)
    x = np.array(b, dtype=np.float64)
    for c in range(N):
        for t in range(4):
            if c + 1 + t < N:
                x[c + 1 + t] -= L[c, t] * x[c]
            if c >= N - 9 and c + 5 + t < N:
                x[c + 5 + t] -= Lw[c, t] * x[c]
    x *= dg
    for c in range(N - 1, -1, -1):
        for t in range(4):
            if c - 1 - t >= 0:
                x[c - 1 - t] -= Uc[c, t] * x[c]
    return x


@pytest.mark.parametrize("N,K,M,m_p", [(16, 3, 3, 1), (33, 2, 4, 2), (48, 2, 3, 2)])
def test_device_factors_solve_the_oracle_operators(opf, N, K, M, m_p):
    """The factors the solve kernel reads (host LU, stored by columns) solve
    the radial operators of section 2.2 as the oracle builds them from its
    own stencils: H_j = 1/dt - c (1/Re)(D2 + D1/r - j^2/r^2 - (alpha k)^2)
    with the Dirichlet wall row, j = m~+1, |m~-1|, m~ for u+, u-, u_z; the
    pressure operator D2 + D1/r - m~^2/r^2 - (alpha k)^2 with the Neumann
    wall row (the (0,0) one with p(1) = 0).  Right-hand sides end in 0 (the
    wall condition), so the check does not depend on how a wall row is
    scaled; normwise backward error against the oracle's matrices."""
    alpha, Re, dt, c = 1.25, 400.0, 0.01, 0.5
    q = lambda what: opf.opf_setup_query(N, K, M, m_p, alpha, Re, dt, what)  # noqa: E731
    luH, luP = q("luH"), q("luP").reshape(K * M + 1, 13 * N)
    hop = q("hop").astype(int).reshape(M, 3)
    nJ = luH.size // (K * 13 * N)
    luH = luH.reshape(K, nJ, 13 * N)
    r = mesh(N)
    mats = {1: fd_matrices(r, 1), -1: fd_matrices(r, -1)}
    rng = np.random.default_rng(11)

    def lap(j, ak, par):
        D1, D2 = mats[par]
        return D2 + D1 / r[:, None] - np.diag(j * j / r ** 2 + ak * ak)

    def check(A, F):
        b = rng.standard_normal(N)
        b[-1] = 0.0
        x = column_substitution(F, b)
        res = np.abs(A @ x - b).max()
        assert res <= 1e-13 * (np.abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max())

    for ik in range(K):
        ak = alpha * ik
        for m in range(M):
            mt = m_p * m
            for f, j in enumerate((mt + 1, abs(mt - 1), mt)):
                H = np.eye(N) / dt - c / Re * lap(j, ak, 1 if j % 2 == 0 else -1)
                H[-1] = 0.0
                H[-1, -1] = 1.0
                check(H, luH[ik, hop[m, f]])
            par = 1 if mt % 2 == 0 else -1
            P = lap(mt, ak, par)
            if ik == 0 and m == 0:
                P[-1] = 0.0
                P[-1, -1] = 1.0
                check(P, luP[K * M])
            else:
                P[-1] = mats[par][0][-1]
                check(P, luP[ik * M + m])
    # the eight-wide lower band lies in the last nine columns only, where the
    # kernel reads it
    for F in list(luH.reshape(-1, 13 * N)) + list(luP):
        assert not np.any(F[4 * N:4 * N + 4 * max(N - 9, 0)])


@pytest.mark.parametrize("N,K,M,m_p", [(16, 3, 3, 1), (33, 2, 4, 2)])
def test_influence_responses_match_the_oracle_operators(opf, N, K, M, m_p):
    """The influence-matrix data of section 2 built by the host, against the
    oracle's operators: per (|k|, m) != (0,0) the pressure p1 with unit wall
    derivative (laplacian 0 inside), the velocity responses to -grad p1
    ((grad p)+- = p' -+ m~ p / r, (grad p)_z = i alpha k p; stored without
    the i), and the responses to unit wall values of u+, u-, u_z; and the
    fixed-flux response G = H_0^{-1} of a uniform forcing (section 1)."""
    alpha, Re, dt, c = 1.25, 400.0, 0.01, 0.5
    q = lambda what: opf.opf_setup_query(N, K, M, m_p, alpha, Re, dt, what)  # noqa: E731
    basis = q("basis").reshape(K, M, 6, N)
    r = mesh(N)
    mats = {1: fd_matrices(r, 1), -1: fd_matrices(r, -1)}
    e = np.zeros(N)
    e[-1] = 1.0

    def lap(j, ak, par):
        D1, D2 = mats[par]
        return D2 + D1 / r[:, None] - np.diag(j * j / r ** 2 + ak * ak)

    def helm_solve(j, ak, rhs):
        H = np.eye(N) / dt - c / Re * lap(j, ak, 1 if j % 2 == 0 else -1)
        H[-1] = 0.0
        H[-1, -1] = 1.0
        return np.linalg.solve(H, rhs)

    for ik in range(K):
        ak = alpha * ik
        for m in range(M):
            if ik == 0 and m == 0:
                assert not np.any(basis[0, 0])
                continue
            mt = m_p * m
            par = 1 if mt % 2 == 0 else -1
            P = lap(mt, ak, par)
            P[-1] = mats[par][0][-1]
            p1 = np.linalg.solve(P, e)
            dp = mats[par][0] @ p1
            rhs = [-(dp - mt * p1 / r), -(dp + mt * p1 / r), -ak * p1]
            for v in rhs:
                v[-1] = 0.0
            js = (mt + 1, abs(mt - 1), mt)
            want = [helm_solve(j, ak, v) for j, v in zip(js, rhs)] + [helm_solve(j, ak, e) for j in js]
            # (the pressure-driven responses against the largest of the three:
            # one of them vanishes where the gradient does, e.g. m~ = 1, k = 0)
            scale_p = max(np.abs(w).max() for w in want[:3])
            for f in range(6):
                scale = scale_p if f < 3 else np.abs(want[f]).max()
                assert np.abs(basis[ik, m, f] - want[f]).max() <= 1e-11 * scale, (ik, m, f)
    g = np.ones(N)
    g[-1] = 0.0
    G = helm_solve(0, 0.0, g)
    assert np.abs(q("G") - G).max() <= 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("N,K,M,m_p", [(16, 3, 3, 1), (33, 2, 4, 2)])
def test_inverse_influence_matrices_match_the_oracle(opf, N, K, M, m_p):
    """The 4 x 4 influence matrices of section 2 per (k, m) != (0,0): column j
    is the boundary vector g = (u+(1), u-(1), u_z(1), div u(1)) of response j
    (the pressure-driven velocity, then unit wall values of u+, u-, u_z), the
    divergence in +- form, 1/2 (u+' + u-') + 1/2 ((1 + m~) u+ + (1 - m~) u-)/r
    + i alpha k u_z, with the oracle's wall stencil of the u+- parity.  The
    host's inverses times the oracle's matrices give the identity."""
    alpha, Re, dt = 1.25, 400.0, 0.01
    q = lambda what: opf.opf_setup_query(N, K, M, m_p, alpha, Re, dt, what)  # noqa: E731
    basis = q("basis").reshape(K, M, 6, N)
    ainv = q("ainv").reshape(M, 2 * K - 1, 4, 4, 2)
    ainv = ainv[..., 0] + 1j * ainv[..., 1]
    r = mesh(N)
    for m in range(M):
        mt = m_p * m
        wall_d1 = fd_matrices(r, -1 if mt % 2 == 0 else 1)[0][-1]  # u+- have parity (-1)^(m~+1)
        for kk in range(2 * K - 1):
            k = kk - (K - 1)
            if k == 0 and m == 0:
                assert not np.any(ainv[m, kk])
                continue
            B = basis[abs(k), m]
            sgn = 1.0 if k >= 0 else -1.0
            resp = [(B[0], B[1], 1j * sgn * B[2]), (B[3], 0 * r, 0 * r), (0 * r, B[4], 0 * r),
                    (0 * r, 0 * r, B[5])]
            A = np.zeros((4, 4), dtype=complex)
            for j, (up, um, uz) in enumerate(resp):
                div = 0.5 * wall_d1 @ (up + um) + 0.5 * ((1 + mt) * up[-1] + (1 - mt) * um[-1]) / r[-1] \
                    + 1j * alpha * k * uz[-1]
                A[:, j] = (up[-1], um[-1], uz[-1], div)
            assert np.abs(ainv[m, kk] @ A - np.eye(4)).max() <= 1e-10, (m, k)


@pytest.mark.parametrize("N,K,M,m_p", [(32, 2, 3, 1), (48, 2, 3, 2)])
def test_split_factors_solve_the_oracle_operators(opf, N, K, M, m_p):
    """The two-partition (split) data of every radial operator: the system
    cut at k = N/2 into diagonal blocks T and B, each substituted on its own
    (device layout), then the interface values z = R (y_T[k-4:k], y_B[0:4])
    and the rank-4 spike corrections x_T = y_T - S_T z_B, x_B = y_B - S_B z_T.
    The result solves the oracle's operators (as in the unsplit check)."""
    alpha, Re, dt, c = 1.25, 400.0, 0.01, 0.5
    q = lambda what: opf.opf_setup_query(N, K, M, m_p, alpha, Re, dt, what)  # noqa: E731
    k = N // 2
    hop = q("hop").astype(int).reshape(M, 3)
    data = {}
    for f in ("H", "P"):
        lu, spk, rr = q("lu" + f + "2"), q("spk" + f), q("r" + f)
        nop = lu.size // (13 * N)
        data[f] = (lu.reshape(nop, 13 * N), spk.reshape(nop, N, 4), rr.reshape(nop, 8, 8))
    nJ = data["H"][0].shape[0] // K
    r = mesh(N)
    mats = {1: fd_matrices(r, 1), -1: fd_matrices(r, -1)}
    rng = np.random.default_rng(5)

    def lap(j, ak, par):
        D1, D2 = mats[par]
        return D2 + D1 / r[:, None] - np.diag(j * j / r ** 2 + ak * ak)

    def check(A, f, o):
        lu, spk, R = (a[o] for a in data[f])
        b = rng.standard_normal(N)
        b[-1] = 0.0
        x = np.empty(N)
        x[:k] = column_substitution(lu[:13 * k], b[:k])
        x[k:] = column_substitution(lu[13 * k:], b[k:])
        z = R @ np.concatenate([x[k - 4:k], x[k:k + 4]])
        x[:k] -= spk[:k] @ z[4:]
        x[k:] -= spk[k:] @ z[:4]
        res = np.abs(A @ x - b).max()
        assert res <= 1e-12 * (np.abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max()), (f, o)

    for ik in range(K):
        ak = alpha * ik
        for m in range(M):
            mt = m_p * m
            for fi, j in enumerate((mt + 1, abs(mt - 1), mt)):
                H = np.eye(N) / dt - c / Re * lap(j, ak, 1 if j % 2 == 0 else -1)
                H[-1] = 0.0
                H[-1, -1] = 1.0
                check(H, "H", ik * nJ + hop[m, fi])
            par = 1 if mt % 2 == 0 else -1
            P = lap(mt, ak, par)
            if ik == 0 and m == 0:
                P[-1] = 0.0
                P[-1, -1] = 1.0
                check(P, "P", K * M)
            else:
                P[-1] = mats[par][0][-1]
                check(P, "P", ik * M + m)


def test_split_arrays_need_an_even_n_of_26_or_more(opf):
    with pytest.raises(opf.OpfError):
        opf.opf_setup_query(25, 2, 2, 1, 1.25, 100.0, 0.01, "luH2")


def test_create_without_a_gpu_fails_with_the_reason(opf):
    """On a machine without a CUDA device the library refuses to create a
    handle and says why (there is no CPU fallback)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(opf.OpfError, match="no CUDA device"):
        opf.opf_create(16, 3, 3, 1, 1.25, 100.0, 0.01)
    with pytest.raises(opf.OpfError, match="need N>=9"):  # arguments are checked first
        opf.opf_create(8, 3, 3, 1, 1.25, 100.0, 0.01)
