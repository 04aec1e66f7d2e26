"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: closed forms,
brute force, a computer-algebra evaluation in Cartesian coordinates, exact
solutions of the Navier-Stokes equations, symmetries, and convergence orders.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sps

from oracle.opf_oracle import Oracle, Params, fd_matrices, mesh, quadrature_weights
from paper_1705_03838_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


# ------------------------------------------------------------------ mesh, FD
def test_mesh_is_half_of_chebyshev_lobatto():
    for N in (9, 16, 33):
        r = mesh(N)
        n = np.arange(1, N + 1)
        # Chebyshev-Lobatto points of degree 2N-1 are where T_(2N-1) = +-1
        T = np.cos((2 * N - 1) * np.arccos(np.clip(r, -1, 1)))
        assert np.allclose(T, (-1.0) ** (N - n), atol=1e-12)
        assert r[-1] == 1.0 and r[0] > 0 and np.all(np.diff(r) > 0)


@pytest.mark.parametrize("parity", [1, -1])
def test_fd_exact_on_polynomials(parity):
    """9-point stencils differentiate polynomials of degree <= 8 exactly
    (section 2), including across the axis with the parity folding."""
    N = 14
    r = mesh(N)
    D1, D2 = fd_matrices(r, parity)
    scale1 = np.abs(D1).sum(axis=1).max()
    scale2 = np.abs(D2).sum(axis=1).max()
    for pw in range(0, 9):
        if (-1) ** pw != parity:
            continue
        f = r ** pw
        d1 = pw * r ** (pw - 1) if pw >= 1 else 0 * r
        d2 = pw * (pw - 1) * r ** (pw - 2) if pw >= 2 else 0 * r
        assert np.abs(D1 @ f - d1).max() <= 1e-13 * scale1
        assert np.abs(D2 @ f - d2).max() <= 1e-13 * scale2


def test_fd_band_structure():
    """Lower bandwidth <= 8 (one-sided wall rows), upper <= 4."""
    N = 20
    D1, D2 = fd_matrices(mesh(N), 1)
    nz = np.argwhere(np.abs(D2) > 0)
    assert (nz[:, 0] - nz[:, 1]).max() == 8
    assert (nz[:, 1] - nz[:, 0]).max() == 4


@pytest.mark.parametrize("parity", [1, -1])
def test_fd_convergence_order(parity):
    g = golden()
    f, d1, d2 = ((lambda r: np.cos(2 * r), lambda r: -2 * np.sin(2 * r), lambda r: -4 * np.cos(2 * r))
                 if parity == 1 else
                 (lambda r: np.sin(2 * r), lambda r: 2 * np.cos(2 * r), lambda r: -4 * np.sin(2 * r)))
    errs = []
    for N in (12, 24):
        r = mesh(N)
        D1, D2 = fd_matrices(r, parity)
        errs.append((np.abs(D1 @ f(r) - d1(r)).max(), np.abs(D2 @ f(r) - d2(r)).max()))
    o1 = math.log2(errs[0][0] / errs[1][0])
    o2 = math.log2(errs[0][1] / errs[1][1])
    assert o1 >= g["d1_order"] - 0.5
    assert o2 >= g["d2_order"] - 0.5


def test_quadrature_exact_and_convergent():
    for N in (9, 16, 40):
        r = mesh(N)
        w = quadrature_weights(r)
        for j in range(4):  # r f with f = r^(2j): degree <= 7 -> exact
            assert abs(w @ r ** (2 * j) - 1.0 / (2 * j + 2)) < 1e-15 * 4
    exact = (math.cos(1.0) + math.sin(1.0) - 1.0)  # int_0^1 r cos r dr
    e16 = abs(quadrature_weights(mesh(16)) @ np.cos(mesh(16)) - exact)
    e32 = abs(quadrature_weights(mesh(32)) @ np.cos(mesh(32)) - exact)
    assert e32 < 1e-12 and e16 < 1e-9


# ------------------------------------------------------------------ user meshes
@pytest.mark.parametrize("parity", [1, -1])
def test_fd_and_quadrature_exact_on_a_user_mesh(parity):
    """Section 2 lets the radial points be supplied: on a mesh clustered
    towards the axis instead of the wall, the 9-point stencils still
    differentiate parity-consistent polynomials of degree <= 8 exactly, and the
    quadrature integrates r f exactly for even f of degree <= 6."""
    N = 18
    r = inputs.stretched_mesh(N)
    assert np.abs(r - mesh(N)).max() > 0.1  # a genuinely different mesh
    D1, D2 = fd_matrices(r, parity)
    s1, s2 = np.abs(D1).sum(axis=1).max(), np.abs(D2).sum(axis=1).max()
    for pw in range(0, 9):
        if (-1) ** pw != parity:
            continue
        d1 = pw * r ** (pw - 1) if pw >= 1 else 0 * r
        d2 = pw * (pw - 1) * r ** (pw - 2) if pw >= 2 else 0 * r
        assert np.abs(D1 @ r ** pw - d1).max() <= 1e-13 * s1
        assert np.abs(D2 @ r ** pw - d2).max() <= 1e-13 * s2
    w = quadrature_weights(r)
    for j in range(4):
        assert abs(w @ r ** (2 * j) - 1.0 / (2 * j + 2)) < 1e-14


def test_steady_and_swirl_solutions_on_a_user_mesh():
    """On the user mesh: Hagen-Poiseuille flow stays steady to round-off and
    the Bessel swirl decays at exp(-j^2 t / Re) to the time and radial
    truncation levels; the mesh reaches every radial operator and the
    quadrature (E = 1 for laminar flow)."""
    N, K, M = 24, 2, 2
    r = inputs.stretched_mesh(N)
    o = Oracle(Params(N, K, M, 1, 1.25, 1000.0, 0.01, r=r))
    lam = inputs.laminar_state(N, K, M, r=r)
    U = o.step(lam, 50)
    assert np.abs(U - lam).max() < 1e-13
    assert np.allclose(o.energy(U), 1.0, atol=1e-13)
    j1 = sps.jn_zeros(1, 1)[0]
    Re, dt, n = 50.0, 0.01, 50
    o = Oracle(Params(N, K, M, 1, 1.25, Re, dt, r=r))
    U0 = lam.copy()
    U0[1, 0, K - 1] = 1e-2 * sps.j1(j1 * r)
    U = o.step(U0, n)
    want = 1e-2 * sps.j1(j1 * r) * math.exp(-j1 ** 2 * n * dt / Re)
    assert np.abs(U[1, 0, K - 1] - want).max() / 1e-2 < 2e-5
    with pytest.raises(ValueError):
        Oracle(Params(N, K, M, 1, 1.25, Re, dt, r=r[::-1]))


# ------------------------------------------------------------------ transforms
def test_dealiased_product_equals_truncated_convolution():
    """3/2 rule (section 2): the pseudo-spectral product of two band-limited
    fields equals the exact convolution, truncated -- by brute force."""
    N, K, M = 9, 3, 4
    p = Params(N, K, M, 1, 1.0, 100.0, 0.01)
    o = Oracle(p)
    rng = np.random.default_rng(3)

    def rand_field():
        A = rng.normal(size=(M, p.nk, N)) + 1j * rng.normal(size=(M, p.nk, N))
        A[0] = 0.5 * (A[0] + np.conj(A[0, ::-1]))
        return A

    A, B = rand_field(), rand_field()
    got = o.analyse(o.synth(A) * o.synth(B))

    def coef(X, k, m):
        if abs(k) >= K or abs(m) >= M:
            return np.zeros(N, complex)
        if m >= 0:
            return X[m, k + K - 1]
        return np.conj(X[-m, -k + K - 1])

    want = np.zeros_like(got)
    for m in range(M):
        for k in range(-(K - 1), K):
            acc = np.zeros(N, complex)
            for k1 in range(-(K - 1), K):
                for m1 in range(-(M - 1), M):
                    acc += coef(A, k1, m1) * coef(B, k - k1, m - m1)
            want[m, k + K - 1] = acc
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_synth_analyse_round_trip():
    N, K, M = 9, 4, 5
    o = Oracle(Params(N, K, M, 1, 1.0, 100.0, 0.01))
    U = inputs.seeded_state(N, K, M, 1, 1.0, 0.1, 7)
    for i in range(3):
        assert np.abs(o.analyse(o.synth(U[i])) - U[i]).max() < 1e-14


# -------------------------------------------- operators vs Cartesian algebra
def _cartesian_case():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    al = sp.Rational(5, 4)
    u = sp.Matrix([
        sp.Rational(3, 10) * y + sp.Rational(1, 5) * x * y * sp.cos(al * z)
        + sp.Rational(1, 7) * (x ** 2 - y ** 2) * sp.sin(al * z),
        -sp.Rational(3, 10) * x + sp.Rational(1, 4) * x ** 2 * sp.sin(al * z)
        + sp.Rational(2, 9) * y * sp.cos(al * z),
        1 - x ** 2 - y ** 2 + sp.Rational(1, 3) * x * sp.cos(al * z)
        + sp.Rational(1, 6) * x * y * sp.sin(al * z),
    ])
    q = x * y * sp.cos(al * z) + sp.Rational(1, 2) * x ** 3 + y * sp.sin(al * z)

    def curl(v):
        return sp.Matrix([sp.diff(v[2], y) - sp.diff(v[1], z),
                          sp.diff(v[0], z) - sp.diff(v[2], x),
                          sp.diff(v[1], x) - sp.diff(v[0], y)])

    def lap(s):
        return sp.diff(s, x, 2) + sp.diff(s, y, 2) + sp.diff(s, z, 2)

    w = curl(u)
    fields = {
        "u": u,
        "omega": w,
        "uxw": u.cross(w),
        "lap": sp.Matrix([lap(u[i]) for i in range(3)]),
        "grad": sp.Matrix([sp.diff(q, x), sp.diff(q, y), sp.diff(q, z)]),
    }
    scalars = {"div": sp.diff(u[0], x) + sp.diff(u[1], y) + sp.diff(u[2], z), "q": q}
    fn = {k: sp.lambdify((x, y, z), list(v), "numpy") for k, v in fields.items()}
    sn = {k: sp.lambdify((x, y, z), v, "numpy") for k, v in scalars.items()}
    return float(al), fn, sn


def _sample(o, fvec, cylindrical=True):
    p = o.p
    th = np.arange(p.nth) * (2 * np.pi / p.m_p) / p.nth
    zz = np.arange(p.nz) * (2 * np.pi / p.alpha) / p.nz
    R, TH, Z = np.meshgrid(o.r, th, zz, indexing="ij")
    X, Y = R * np.cos(TH), R * np.sin(TH)
    vals = [np.broadcast_to(np.asarray(v, dtype=float), X.shape) for v in fvec(X, Y, Z)]
    vr = vals[0] * np.cos(TH) + vals[1] * np.sin(TH)
    vt = -vals[0] * np.sin(TH) + vals[1] * np.cos(TH)
    out = [vr, vt, vals[2]]
    # oracle physical layout is (N, nz, nth)
    return [np.transpose(c, (0, 2, 1)) for c in out]


def _sample_scalar(o, f):
    p = o.p
    th = np.arange(p.nth) * (2 * np.pi / p.m_p) / p.nth
    zz = np.arange(p.nz) * (2 * np.pi / p.alpha) / p.nz
    R, TH, Z = np.meshgrid(o.r, th, zz, indexing="ij")
    v = np.broadcast_to(np.asarray(f(R * np.cos(TH), R * np.sin(TH), Z), dtype=float), R.shape)
    return np.transpose(v, (0, 2, 1))


def test_operators_match_cartesian_calculus():
    """curl, div, grad, vector Laplacian and u x omega of the oracle equal the
    Cartesian computer-algebra values on a polynomial field (exact for 9-point
    FD), projected onto (r, theta, z)."""
    al, fn, sn = _cartesian_case()
    p = Params(12, 3, 7, 1, al, 100.0, 0.01)
    o = Oracle(p)

    def spec(name):
        return np.stack([o.analyse(c) for c in _sample(o, fn[name])])

    U = spec("u")
    tol = 1e-10
    assert np.abs(o.curl(U) - spec("omega")).max() < tol
    assert np.abs(o.vector_laplacian(U) - spec("lap")).max() < 1e-8
    assert np.abs(o.divergence(U) - o.analyse(_sample_scalar(o, sn["div"]))).max() < tol
    Q = o.analyse(_sample_scalar(o, sn["q"]))
    assert np.abs(o.gradient(Q) - spec("grad")).max() < tol
    Nl = o.nonlinear(U)
    Nl[2, 0, p.K - 1] -= 4.0 / p.Re
    assert np.abs(Nl - spec("uxw")).max() < tol


# ------------------------------------------------------- whole-step: exact flows
def test_hagen_poiseuille_is_steady():
    p = Params(16, 4, 4, 1, 1.25, 2000.0, 0.01)
    o = Oracle(p)
    U0 = inputs.laminar_state(16, 4, 4)
    U = o.step(U0, 100)
    assert np.abs(U - U0).max() < 1e-13
    assert abs(o.beta) * 4.0 / p.Re < 1e-13  # beta' (forcing increment)
    assert np.allclose(o.energy(U), 1.0, atol=1e-13)


def _swirl(N, K, M, eps, j1):
    U = inputs.laminar_state(N, K, M)
    r = mesh(N)
    U[1, 0, K - 1] = eps * sps.j1(j1 * r)
    return U


def test_bessel_swirl_decays_at_exact_rate():
    """u_theta = J1(j r) on top of Hagen-Poiseuille is an exact solution;
    it decays as exp(-j^2 t / Re).  The c = 1/2 scheme is 2nd order in dt."""
    j1 = sps.jn_zeros(1, 1)[0]
    N, K, M, Re = 24, 2, 2, 50.0
    errs = []
    for dt, n in ((0.02, 25), (0.01, 50)):
        o = Oracle(Params(N, K, M, 1, 1.25, Re, dt))
        U = o.step(_swirl(N, K, M, 1e-2, j1), n)
        t = dt * n
        want = 1e-2 * sps.j1(j1 * o.r) * math.exp(-j1 ** 2 * t / Re)
        errs.append(np.abs(U[1, 0, K - 1] - want).max() / 1e-2)
        # the discrete grad p matches u x omega only to truncation level, so the
        # axial flow feels the swirl at that level (N = 24: ~1e-11)
        assert np.abs(U[2, 0, K - 1] - (1 - o.r ** 2)).max() < 1e-9
    assert errs[1] < 2e-6
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_swirl_amplitude_per_step_follows_the_theta_method_at_c_not_half():
    """Implicitness c != 1/2 with two correctors: u x omega of the swirl is a
    pure radial gradient, so every corrector leaves the viscous update alone
    and each step multiplies the swirl by the theta-method factor
    g = (1 + (1-c) lambda dt) / (1 - c lambda dt), lambda = -j^2/Re
    (section 2: c weights the implicit viscous term).  At c = 0.6 g^n differs
    from exp(lambda t) by ~(c - 1/2) lambda^2 dt t = 4e-5; the closed form
    holds to the spatial truncation level (~1e-9 at N = 24)."""
    j1 = sps.jn_zeros(1, 1)[0]
    N, K, M, Re, dt, n, c = 24, 2, 2, 50.0, 0.01, 50, 0.6
    o = Oracle(Params(N, K, M, 1, 1.25, Re, dt, c=c, n_corr=2))
    U = o.step(_swirl(N, K, M, 1e-2, j1), n)
    lam = -j1 ** 2 / Re
    g = (1 + (1 - c) * lam * dt) / (1 - c * lam * dt)
    shape = 1e-2 * sps.j1(j1 * o.r)
    err_theta = np.abs(U[1, 0, K - 1] - g ** n * shape).max() / 1e-2
    err_exp = np.abs(U[1, 0, K - 1] - math.exp(lam * n * dt) * shape).max() / 1e-2
    assert err_theta < 2e-8
    assert err_exp > 1e-5  # the c = 0.6 scheme is not second order


def _time_refinement(c, n_corr, dts, ref, U0, T, args):
    errs = []
    lam = inputs.laminar_state(args[0], args[1], args[2])
    for dt in dts:
        U = Oracle(Params(*args, dt, c=c, n_corr=n_corr)).step(U0, int(round(T / dt)))
        errs.append(np.linalg.norm(U - ref) / np.linalg.norm(ref - lam))
    return errs


@pytest.fixture(scope="module")
def refinement_case():
    """A nonlinear run (amplitude 0.3, Re = 5000, N = 12) to T = 0.4, and a
    reference at dt = 0.05/64 shared by every scheme below."""
    args = (12, 3, 3, 1, 1.25, 5000.0)
    U0 = inputs.seeded_state(12, 3, 3, 1, 1.25, 0.3, 31)
    T, dtr = 0.4, 0.05 / 64
    ref = Oracle(Params(*args, dtr, n_corr=3)).step(U0, int(round(T / dtr)))
    return args, U0, T, ref


@pytest.mark.parametrize("c,n_corr,lo,hi", [(0.5, 1, 1.7, 2.5), (0.5, 2, 1.7, 2.5),
                                            (0.6, 1, 0.8, 1.25), (0.6, 2, 0.8, 1.25)])
def test_time_refinement_order_of_the_predictor_corrector(refinement_case, c, n_corr, lo, hi):
    """Section 2's predictor-corrector: second order at c = 1/2 with one or
    two corrector iterations, first order at c = 0.6 (weights c, 1 - c on
    both the viscous and the nonlinear term).  Every scheme converges to the
    same limit, so the weights of each term sum to one.  A corrector that
    took N from u_j instead of from the latest iterate would fall to first
    order at n_corr = 2; a nonlinear weight pair that did not sum to one
    would stall against the common reference."""
    args, U0, T, ref = refinement_case
    errs = _time_refinement(c, n_corr, (0.025, 0.0125, 0.00625), ref, U0, T, args)
    order = math.log2(errs[1] / errs[2])
    assert lo < order < hi, (errs, order)
    assert errs[2] < (5e-5 if c == 0.5 else 5e-4)


@pytest.mark.parametrize("c,n_corr", [(0.6, 1), (0.4, 2)])
def test_first_order_error_constant_of_the_theta_weights(c, n_corr):
    """With both the viscous and the nonlinear term weighted c (new level) and
    1 - c (old level), the local error of a step is (c - 1/2) dt^2 u'' + O(dt^3),
    so over a short time T the global error is (c - 1/2) dt (u'(T) - u'(0))
    to leading order.  u' comes from a fine reference trajectory by one-sided
    differences, the O(dt^2) part of the error is removed by Richardson
    extrapolation over dt and dt/2.  Swapping the two nonlinear weights keeps
    the scheme consistent and first order but flips the sign of the
    (dominant) advective part of this error: the cosine goes to ~ -0.9."""
    args = (12, 3, 3, 1, 1.25, 5000.0)
    U0 = inputs.seeded_state(12, 3, 3, 1, 1.25, 0.3, 31)
    T, dtr = 0.05, 0.05 / 400
    o = Oracle(Params(*args, dtr, n_corr=3))
    traj = [U0]
    for _ in range(int(round(T / dtr))):
        traj.append(o.step(traj[-1], 1))
    ud0 = (-3 * traj[0] + 4 * traj[1] - traj[2]) / (2 * dtr)
    udT = (3 * traj[-1] - 4 * traj[-2] + traj[-3]) / (2 * dtr)
    pred = (c - 0.5) * (udT - ud0)
    es = []
    for dt in (0.005, 0.0025):
        V = Oracle(Params(*args, dt, c=c, n_corr=n_corr)).step(U0, int(round(T / dt)))
        es.append((V - traj[-1]) / dt)
    e = 2 * es[1] - es[0]
    cos = np.real(np.vdot(e, pred)) / (np.linalg.norm(e) * np.linalg.norm(pred))
    ratio = np.linalg.norm(e) / np.linalg.norm(pred)
    assert cos > 0.7 and 0.8 < ratio < 1.25, (cos, ratio)


def test_linear_limit_is_quadratic_in_the_amplitude():
    """Hagen-Poiseuille is a fixed point of the step and u x w is quadratic,
    so a step from u_lam + eps v gives (S - u_lam)/eps = A v + eps B(v) +
    O(eps^2): halving eps halves the difference of successive quotients.  A
    stray constant term (a wrong driving force) or a cubic one breaks the
    ratio 2."""
    N, K, M, m_p, alpha, Re, dt = 16, 3, 3, 1, 1.25, 500.0, 0.01
    lam = inputs.laminar_state(N, K, M)
    v = inputs.seeded_state(N, K, M, m_p, alpha, 1.0, 5, laminar=False)
    o = Oracle(Params(N, K, M, m_p, alpha, Re, dt))
    q = [(o.step(lam + eps * v, 3) - lam) / eps for eps in (1e-2, 5e-3, 2.5e-3, 1.25e-3)]
    d = [np.linalg.norm(q[i] - q[i + 1]) for i in range(3)]
    assert d[0] > 1e-6 * np.linalg.norm(q[0])  # the nonlinear term is there
    assert abs(d[0] / d[1] - 2.0) < 2e-3 and abs(d[1] / d[2] - 2.0) < 2e-3


def test_radial_refinement_of_the_step():
    """Two steps from one smooth field on N = 16 ... 40 radial points (the
    field and the results moved between meshes by the 9-point interpolation,
    itself exact on polynomials) against N = 64: the error falls
    monotonically and reaches the order of the 9-point stencils (section 2:
    orders 8 and 7) by N = 32 ... 40."""
    from oracle.opf_oracle import change_resolution

    K, M, alpha, Re, dt, NF = 3, 3, 1.25, 500.0, 0.01, 64
    U0 = inputs.seeded_state(NF, K, M, 1, alpha, 0.05, 9)
    ref = Oracle(Params(NF, K, M, 1, alpha, Re, dt)).step(U0, 2)
    scale = np.linalg.norm(ref - inputs.laminar_state(NF, K, M))
    Ns = (16, 24, 32, 40)
    errs = []
    for n in Ns:
        U = Oracle(Params(n, K, M, 1, alpha, Re, dt)).step(change_resolution(U0, n, K, M, 1), 2)
        errs.append(np.linalg.norm(change_resolution(U, NF, K, M, 1) - ref) / scale)
    assert all(errs[i + 1] < errs[i] for i in range(3))
    order = math.log(errs[2] / errs[3]) / math.log(Ns[3] / Ns[2])
    assert order > 5.5, (errs, order)


def test_solve_restricted_to_modes_equals_the_full_solve():
    """solve_modes (used to check grids too large for the dense solve of
    every mode) gives exactly the full solve's modes and beta'."""
    o = Oracle(Params(12, 3, 4, 1, 1.25, 500.0, 0.01))
    U = inputs.seeded_state(12, 3, 4, 1, 1.25, 0.1, 3)
    Nj = o.nonlinear(U)
    full, bp = o.solve(U, Nj)
    for (m, kk), (u, b) in o.solve_modes(U, Nj, [(0, 2), (1, 0), (3, 4), (2, 2)]).items():
        assert np.array_equal(u, full[:, m, kk])
        assert b == (bp if (m, kk) == (0, 2) else 0.0)


def test_wall_conditions_at_round_off():
    """||g|| (no-slip and wall divergence) at machine epsilon (section 2)."""
    N, K, M = 16, 4, 4
    o = Oracle(Params(N, K, M, 1, 1.25, 1000.0, 0.01))
    U = o.step(inputs.seeded_state(N, K, M, 1, 1.25, 0.05, 11), 5)
    g_u, g_div = o.wall_residual(U)
    assert g_u < 1e-15
    assert g_div < 1e-11
    assert abs(2 * np.pi * (U[2, 0, K - 1].real @ o.w) - np.pi / 2) < 1e-14


# ------------------------------------------------------------- symmetries
def test_rotational_symmetry_m_p():
    """m_p = 2 with M modes equals m_p = 1 with 2M-1 modes, odd ones zero."""
    N, K, M = 12, 3, 3
    a = Oracle(Params(N, K, M, 2, 1.25, 500.0, 0.01))
    b = Oracle(Params(N, K, 2 * M - 1, 1, 1.25, 500.0, 0.01))
    Ua = inputs.seeded_state(N, K, M, 2, 1.25, 0.05, 5)
    Ub = np.zeros((3, 2 * M - 1, 2 * K - 1, N), complex)
    Ub[:, 0::2] = Ua
    Va = a.step(Ua, 3)
    Vb = b.step(Ub, 3)
    assert np.abs(Vb[:, 0::2] - Va).max() < 1e-12
    assert np.abs(Vb[:, 1::2]).max() < 1e-15
    assert np.allclose(a.energy(Va), b.energy(Vb), rtol=1e-12)


def test_axial_shift_equivariance():
    N, K, M = 12, 4, 3
    alpha = 1.25
    o = Oracle(Params(N, K, M, 1, alpha, 500.0, 0.01))
    U = inputs.seeded_state(N, K, M, 1, alpha, 0.05, 9)
    shift = np.exp(1j * alpha * np.arange(-(K - 1), K) * 0.7)[None, None, :, None]
    A = o.step(U * shift, 2)
    B = o.step(U, 2) * shift
    assert np.abs(A - B).max() < 1e-13


def test_perturbations_travel_downstream():
    """Small disturbances are carried by the mean flow: phase speed in (0, 1)."""
    N, K, M = 16, 2, 2
    alpha = 1.0
    o = Oracle(Params(N, K, M, 1, alpha, 1000.0, 0.01))
    U0 = inputs.laminar_state(N, K, M)
    pert = inputs.seeded_state(N, K, M, 1, alpha, 1e-6, 21, laminar=False)
    pert[:, :, K - 1] = 0.0  # k = 0 parts do not travel
    U = o.step(U0 + pert, 50)
    d0 = pert[:, 1, K]  # k = +1, m = 1
    d1 = (U - U0)[:, 1, K]
    phase = np.angle(np.vdot(d0, d1))  # ~ -alpha c t
    t = 0.5
    assert -alpha * t < phase < -0.05 * alpha * t


# ------------------------------------------------------------- energy E, I, D
def test_energy_budget():
    """dE/dt = I - D; with laminar normalisation dE^/dt = (12/Re)(I^ - D^)."""
    N, K, M, Re, dt = 24, 4, 4, 500.0, 0.002
    o = Oracle(Params(N, K, M, 1, 1.25, Re, dt))
    U = inputs.seeded_state(N, K, M, 1, 1.25, 0.1, 13)
    U = o.step(U, 5)
    e0 = o.energy(U)
    U = o.step(U, 1)
    e1 = o.energy(U)
    U = o.step(U, 1)
    e2 = o.energy(U)
    lhs = (e2[0] - e0[0]) / (2 * dt)
    rhs = (12.0 / Re) * (e1[1] - e1[2])
    assert abs(lhs - rhs) < 1e-3 * abs(12.0 / Re * e1[2])


def test_paper_growth_factor_is_consistent():
    """Section 3.2: eigenvalue 0.00620 + 0.0183i grows by 8.4 per rotation
    (arithmetic consistency of the printed values; the state is not available)."""
    g = golden()
    growth = math.exp(g["n2ml_eig_re"] * 2 * math.pi / g["n2ml_eig_im"])
    assert abs(growth - g["n2ml_growth"]) < 0.05
