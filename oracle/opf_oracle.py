"""Plain, slow FP64 CPU oracle for the pipe-flow time step of Openpipeflow
(Willis 2017, "The Openpipeflow Navier-Stokes solver").

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference arm may import this module.  The CUDA library never
calls it, and it shares no code with the CUDA path: it is written from the
paper's description plus textbook cylindrical Navier-Stokes, with the most
direct numerics available:

  * finite-difference weights as derivatives of the 9-point Lagrange
    interpolant, written out as sums of products (no recursion);
  * Eq. 1 synthesised/analysed with numpy's 2-D FFT on the 3K x 3M grid;
  * the full product u x omega of the TOTAL velocity;
  * per Fourier mode, one dense complex linear system in the unknowns
    (u_r, u_theta, u_z, p [, beta']) -- implicit momentum, pressure-Poisson
    equation, and the four boundary conditions g = 0 imposed directly as
    rows -- solved by LU with partial pivoting (LAPACK via scipy).  This is
    the system the influence-matrix technique solves (paper section 2); the
    oracle does not use influence matrices or the u+/u- decoupling.

State layout: complex128 (3, M, 2K-1, N) = (u_r, u_theta, u_z)[m][k+K-1][n],
total velocity, r_N = 1 the wall.

Readings of points the paper leaves open (each is a choice, stated here):
  R1 mesh: r_n = cos(pi (N-n)/(2N-1)), the positive half of 2N Chebyshev-
     Lobatto points (includes the wall, excludes the axis);
  R2 Eq. 1 index ranges: |k| < K, 0 <= m < M, negative m by conjugation;
  R3 stencils: the 9 index-nearest points of {-r_N..-r_1, r_1..r_N}, shifted
     inward at the wall; values at -r_j folded onto r_j with the field's axis
     parity, (-1)^m~ for u_z and p, (-1)^(m~+1) for u_r, u_theta;
  R4 implicitness c weights both the viscous term and the corrector's
     nonlinear term; one corrector iteration;
  R5 PPE: lap p = div(N_eff), N_eff = c N^q + (1-c) N_j; the wall-divergence
     condition closes it; the (0,0) mode uses the gauge p(1) = 0;
  R6 fixed flux: a uniform extra axial forcing beta' in the implicit
     equation of the (0,0) mode, chosen so 2 pi int u_z r dr = pi/2;
     reported beta = beta' Re / 4 (forcing (4/Re)(1 + beta));
  R7 quadrature: int_0^1 f r dr by integrating the 9-point interpolant of
     r f over each interval [r_(n-1), r_n] (r_0 = 0) with row n's stencil.
"""

import numpy as np
import scipy.linalg as sla

__all__ = [
    "Params", "mesh", "lagrange_weights", "fd_matrices", "quadrature_weights",
    "Oracle",
]


class Params:
    """Run parameters (paper section 2): resolution (N, K, M), m_p, alpha, Re, dt."""

    def __init__(self, N, K, M, m_p, alpha, Re, dt, c=0.5, n_corr=1, rotation=(0.0, 0.0, 0.0), forcing=None,
                 r=None):
        self.N, self.K, self.M, self.m_p = int(N), int(K), int(M), int(m_p)
        # r: a user radial mesh (section 2: the points may be read from a
        # file instead of the default formula), N increasing points in (0, 1]
        # with the wall r_N = 1; None = reading R1's points
        self.r = None if r is None else np.array(r, dtype=np.float64)
        self.alpha, self.Re, self.dt = float(alpha), float(Re), float(dt)
        self.c, self.n_corr = float(c), int(n_corr)
        # frame rotation Omega (Cartesian, pipe axis z): Coriolis force -2 Omega x u
        # (section 3.1 adds it through the forcing hook); forcing: a constant
        # spectral body force (3, M, 2K-1, N) in (r, theta, z) components
        self.rotation = tuple(float(x) for x in rotation)
        self.forcing = forcing
        self.nk = 2 * self.K - 1
        self.nz = 3 * self.K  # 3/2 dealiasing: 3K x 3M grid (section 2)
        self.nth = 3 * self.M


# ---------------------------------------------------------------- radial mesh
def mesh(N):
    """Radial points (section 2, reading R1)."""
    n = np.arange(1, N + 1, dtype=np.float64)
    return np.cos(np.pi * (N - n) / (2 * N - 1))


def lagrange_weights(x0, nodes):
    """First and second derivative at x0 of each Lagrange basis polynomial
    l_i(x) = prod_{j != i} (x - x_j)/(x_i - x_j), by the product rule."""
    n = len(nodes)
    w1 = np.zeros(n)
    w2 = np.zeros(n)
    for i in range(n):
        others = [j for j in range(n) if j != i]
        s1 = 0.0
        s2 = 0.0
        for a in others:
            pa = 1.0 / (nodes[i] - nodes[a])
            prod = 1.0
            for j in others:
                if j != a:
                    prod *= (x0 - nodes[j]) / (nodes[i] - nodes[j])
            s1 += pa * prod
            for b in others:
                if b == a:
                    continue
                pb = 1.0 / (nodes[i] - nodes[b])
                prod2 = 1.0
                for j in others:
                    if j != a and j != b:
                        prod2 *= (x0 - nodes[j]) / (nodes[i] - nodes[j])
                s2 += pa * pb * prod2
        w1[i] = s1
        w2[i] = s2
    return w1, w2


def _stencil(N, n):
    """Extended-set indices of row n's 9-point stencil (reading R3).
    Extended set E (sorted): E[e] = -r[N-1-e] for e < N, r[e-N] for e >= N."""
    q = N + n
    lo, hi = q - 4, q + 4
    if hi > 2 * N - 1:
        lo, hi = 2 * N - 9, 2 * N - 1
    return list(range(lo, hi + 1))


def _extended(r):
    return np.concatenate([-r[::-1], r])


def _fold(N, e, parity):
    """Column and sign that extended index e folds onto."""
    if e >= N:
        return e - N, 1.0
    return N - 1 - e, float(parity)


def fd_matrices(r, parity):
    """Dense N x N first/second radial derivative matrices (9 points, section 2)
    for a field of axis parity `parity` (+1 even, -1 odd)."""
    N = len(r)
    ext = _extended(r)
    D1 = np.zeros((N, N))
    D2 = np.zeros((N, N))
    for n in range(N):
        idx = _stencil(N, n)
        w1, w2 = lagrange_weights(r[n], ext[idx])
        for t, e in enumerate(idx):
            col, sgn = _fold(N, e, parity)
            D1[n, col] += sgn * w1[t]
            D2[n, col] += sgn * w2[t]
    return D1, D2


def quadrature_weights(r):
    """w with sum_n w_n f(r_n) ~ int_0^1 f(r) r dr for even f (reading R7)."""
    N = len(r)
    ext = _extended(r)
    gx, gw = np.polynomial.legendre.leggauss(8)
    w = np.zeros(N)
    for n in range(N):
        a = 0.0 if n == 0 else r[n - 1]
        b = r[n]
        xs = 0.5 * (b - a) * gx + 0.5 * (a + b)
        ws = 0.5 * (b - a) * gw
        idx = _stencil(N, n)
        nodes = ext[idx]
        for t, e in enumerate(idx):
            lt = np.ones_like(xs)
            for s, x_s in enumerate(nodes):
                if s != t:
                    lt *= (xs - x_s) / (nodes[t] - x_s)
            integral = float(np.sum(ws * lt))
            col, _ = _fold(N, e, 1.0)
            w[col] += integral * ext[e]  # value of r f at the node, f even
    return w


# --------------------------------------------------------------------- oracle
class Oracle:
    """The time step of section 2 for one parameter set."""

    def __init__(self, p: Params):
        self.p = p
        N = p.N
        if N < 9:
            raise ValueError("need N >= 9 for the 9-point stencil")
        if p.r is None:
            self.r = mesh(N)
        else:
            r = p.r
            if r.shape != (N,) or not (r[0] > 0 and r[-1] == 1.0 and np.all(np.diff(r) > 0)):
                raise ValueError("a user mesh needs N increasing points in (0, 1] ending at the wall r = 1")
            self.r = r.copy()
        self.D = {s: fd_matrices(self.r, s) for s in (1, -1)}
        self.w = quadrature_weights(self.r)
        self._lu = {}
        self.beta = 0.0

    # ---- helpers
    def mt(self, m):
        return self.p.m_p * m

    def ak(self, kk):
        return self.p.alpha * (kk - (self.p.K - 1))

    def par_s(self, m):
        """Axis parity of u_z and p for azimuthal index m."""
        return 1 if self.mt(m) % 2 == 0 else -1

    def par_v(self, m):
        """Axis parity of u_r and u_theta."""
        return -self.par_s(m)

    def scalar_laplacian(self, m, kk, parity):
        D1, D2 = self.D[parity]
        r = self.r
        return D2 + np.diag(1.0 / r) @ D1 - np.diag(self.mt(m) ** 2 / r ** 2 + self.ak(kk) ** 2)

    # ---- spectral differential operators (cylindrical, textbook)
    def curl(self, U):
        p, r = self.p, self.r
        W = np.zeros_like(U)
        for m in range(p.M):
            mt = self.mt(m)
            D1v = self.D[self.par_v(m)][0]
            D1s = self.D[self.par_s(m)][0]
            for kk in range(p.nk):
                ak = self.ak(kk)
                ur, ut, uz = U[0, m, kk], U[1, m, kk], U[2, m, kk]
                W[0, m, kk] = 1j * mt * uz / r - 1j * ak * ut
                W[1, m, kk] = 1j * ak * ur - D1s @ uz
                W[2, m, kk] = D1v @ ut + ut / r - 1j * mt * ur / r
        return W

    def divergence(self, U):
        p, r = self.p, self.r
        out = np.zeros(U.shape[1:], dtype=np.complex128)
        for m in range(p.M):
            mt = self.mt(m)
            D1v = self.D[self.par_v(m)][0]
            for kk in range(p.nk):
                ak = self.ak(kk)
                out[m, kk] = (D1v @ U[0, m, kk] + U[0, m, kk] / r
                              + 1j * mt * U[1, m, kk] / r + 1j * ak * U[2, m, kk])
        return out

    def gradient(self, P):
        p, r = self.p, self.r
        G = np.zeros((3,) + P.shape, dtype=np.complex128)
        for m in range(p.M):
            mt = self.mt(m)
            D1s = self.D[self.par_s(m)][0]
            for kk in range(p.nk):
                G[0, m, kk] = D1s @ P[m, kk]
                G[1, m, kk] = 1j * mt * P[m, kk] / r
                G[2, m, kk] = 1j * self.ak(kk) * P[m, kk]
        return G

    def vector_laplacian(self, U):
        """Components of lap(u) in cylindrical coordinates."""
        p, r = self.p, self.r
        L = np.zeros_like(U)
        for m in range(p.M):
            mt = self.mt(m)
            for kk in range(p.nk):
                Lv = self.scalar_laplacian(m, kk, self.par_v(m))
                Ls = self.scalar_laplacian(m, kk, self.par_s(m))
                ur, ut, uz = U[0, m, kk], U[1, m, kk], U[2, m, kk]
                L[0, m, kk] = Lv @ ur - ur / r ** 2 - 2j * mt * ut / r ** 2
                L[1, m, kk] = Lv @ ut - ut / r ** 2 + 2j * mt * ur / r ** 2
                L[2, m, kk] = Ls @ uz
        return L

    # ---- Eq. 1 on the 3K x 3M grid
    def synth(self, A):
        """Physical values (N, 3K, 3M) of a spectral scalar (M, 2K-1, N), Eq. 1."""
        p = self.p
        C = np.zeros((p.N, p.nz, p.nth), dtype=np.complex128)
        for kk in range(p.nk):
            k = kk - (p.K - 1)
            # m = 0: real field, take the Hermitian part of the k-pair
            C[:, k % p.nz, 0] = 0.5 * (A[0, kk] + np.conj(A[0, p.nk - 1 - kk]))
            for m in range(1, p.M):
                C[:, k % p.nz, m] = A[m, kk]
                C[:, (-k) % p.nz, (-m) % p.nth] = np.conj(A[m, kk])
        phys = np.fft.ifft2(C, axes=(1, 2), norm="forward")
        return phys.real

    def analyse(self, phys):
        """Truncated spectral coefficients (M, 2K-1, N) of a physical scalar."""
        p = self.p
        C = np.fft.fft2(phys, axes=(1, 2), norm="forward")
        A = np.zeros((p.M, p.nk, p.N), dtype=np.complex128)
        for kk in range(p.nk):
            k = kk - (p.K - 1)
            for m in range(p.M):
                A[m, kk] = C[:, k % p.nz, m]
        return A

    def nonlinear(self, U):
        """u x omega evaluated pseudo-spectrally, plus the base forcing 4/Re."""
        W = self.curl(U)
        u = [self.synth(U[i]) for i in range(3)]
        w = [self.synth(W[i]) for i in range(3)]
        n_r = u[1] * w[2] - u[2] * w[1]
        n_t = u[2] * w[0] - u[0] * w[2]
        n_z = u[0] * w[1] - u[1] * w[0]
        ox, oy, oz = self.p.rotation
        if ox or oy or oz:
            # Omega in cylindrical components at theta = 2 pi q / (m_p 3M)
            th = 2.0 * np.pi * np.arange(self.p.nth) / (self.p.m_p * self.p.nth)
            o_r = (ox * np.cos(th) + oy * np.sin(th))[None, None, :]
            o_t = (-ox * np.sin(th) + oy * np.cos(th))[None, None, :]
            n_r = n_r - 2.0 * (o_t * u[2] - oz * u[1])
            n_t = n_t - 2.0 * (oz * u[0] - o_r * u[2])
            n_z = n_z - 2.0 * (o_r * u[1] - o_t * u[0])
        Nl = np.stack([self.analyse(n_r), self.analyse(n_t), self.analyse(n_z)])
        Nl[2, 0, self.p.K - 1] += 4.0 / self.p.Re
        if self.p.forcing is not None:
            Nl = Nl + self.p.forcing
        return Nl

    # ---- implicit solve, one dense system per mode
    def _mode_matrix(self, m, kk):
        p, r = self.p, self.r
        N, c, nu, dt = p.N, p.c, 1.0 / p.Re, p.dt
        mt, ak = self.mt(m), self.ak(kk)
        mean = (m == 0 and kk == p.K - 1)
        size = 4 * N + (1 if mean else 0)
        A = np.zeros((size, size), dtype=np.complex128)
        I = np.eye(N)
        R1 = np.diag(1.0 / r)
        R2 = np.diag(1.0 / r ** 2)
        Lv = self.scalar_laplacian(m, kk, self.par_v(m))
        Ls = self.scalar_laplacian(m, kk, self.par_s(m))
        D1s = self.D[self.par_s(m)][0]
        D1v = self.D[self.par_v(m)][0]
        sr, st, sz, sp = slice(0, N), slice(N, 2 * N), slice(2 * N, 3 * N), slice(3 * N, 4 * N)
        A[sr, sr] = I / dt - c * nu * (Lv - R2)
        A[sr, st] = -c * nu * (-2j * mt * R2)
        A[sr, sp] = D1s
        A[st, sr] = -c * nu * (2j * mt * R2)
        A[st, st] = I / dt - c * nu * (Lv - R2)
        A[st, sp] = 1j * mt * R1
        A[sz, sz] = I / dt - c * nu * Ls
        A[sz, sp] = 1j * ak * I
        A[sp, sp] = Ls
        w = N - 1
        for blk in (0, 1, 2):  # no-slip rows
            A[blk * N + w, :] = 0.0
            A[blk * N + w, blk * N + w] = 1.0
        A[3 * N + w, :] = 0.0
        if mean:
            A[3 * N + w, 3 * N + w] = 1.0  # gauge p(1) = 0
            A[2 * N: 2 * N + w, 4 * N] = -1.0  # extra uniform forcing beta'
            A[4 * N, sz] = 2.0 * np.pi * self.w
        else:  # wall divergence = 0
            A[3 * N + w, sr] = D1v[w]
            A[3 * N + w, w] += 1.0 / r[w]
            A[3 * N + w, N + w] += 1j * mt / r[w]
            A[3 * N + w, 2 * N + w] += 1j * ak
        return A

    def _lu_factor(self, m, kk):
        key = (m, kk)
        if key not in self._lu:
            self._lu[key] = sla.lu_factor(self._mode_matrix(m, kk))
        return self._lu[key]

    def solve(self, Uj, Neff):
        """u with (1/dt - c L)u + grad p = (1/dt + (1-c)L)u_j + N_eff,
        lap p = div N_eff, g = 0; also returns beta'."""
        p = self.p
        N, c, nu, dt = p.N, p.c, 1.0 / p.Re, p.dt
        Lu = self.vector_laplacian(Uj)
        R = Uj / dt + (1.0 - c) * nu * Lu + Neff
        dN = self.divergence(Neff)
        Unew = np.zeros_like(Uj)
        beta_p = 0.0
        for m in range(p.M):
            for kk in range(p.nk):
                mean = (m == 0 and kk == p.K - 1)
                b = np.zeros(4 * N + (1 if mean else 0), dtype=np.complex128)
                for blk in range(3):
                    b[blk * N: (blk + 1) * N] = R[blk, m, kk]
                    b[blk * N + N - 1] = 0.0
                b[3 * N: 4 * N] = dN[m, kk]
                b[4 * N - 1] = 0.0
                if mean:
                    b[4 * N] = np.pi / 2.0
                x = sla.lu_solve(self._lu_factor(m, kk), b)
                for blk in range(3):
                    Unew[blk, m, kk] = x[blk * N: (blk + 1) * N]
                if mean:
                    beta_p = x[4 * N].real
        return Unew, beta_p

    def solve_modes(self, Uj, Neff, modes):
        """solve() restricted to the listed (m, kk) modes: each mode's system
        involves only that mode's u_j and N_eff, so grids too large for a
        dense solve of every mode can still be checked mode by mode.  Returns
        {(m, kk): (u (3, N), beta')}, with the same right-hand side and dense
        system as solve()."""
        p, r = self.p, self.r
        N, c, nu, dt = p.N, p.c, 1.0 / p.Re, p.dt
        out = {}
        for m, kk in modes:
            mt, ak = self.mt(m), self.ak(kk)
            Lv = self.scalar_laplacian(m, kk, self.par_v(m))
            Ls = self.scalar_laplacian(m, kk, self.par_s(m))
            ur, ut, uz = Uj[0, m, kk], Uj[1, m, kk], Uj[2, m, kk]
            Lu = np.stack([Lv @ ur - ur / r ** 2 - 2j * mt * ut / r ** 2,
                           Lv @ ut - ut / r ** 2 + 2j * mt * ur / r ** 2,
                           Ls @ uz])
            R = Uj[:, m, kk] / dt + (1.0 - c) * nu * Lu + Neff[:, m, kk]
            D1v = self.D[self.par_v(m)][0]
            nr, nt, nz = Neff[0, m, kk], Neff[1, m, kk], Neff[2, m, kk]
            dN = D1v @ nr + nr / r + 1j * mt * nt / r + 1j * ak * nz
            mean = (m == 0 and kk == p.K - 1)
            b = np.zeros(4 * N + (1 if mean else 0), dtype=np.complex128)
            for blk in range(3):
                b[blk * N: (blk + 1) * N] = R[blk]
                b[blk * N + N - 1] = 0.0
            b[3 * N: 4 * N] = dN
            b[4 * N - 1] = 0.0
            if mean:
                b[4 * N] = np.pi / 2.0
            x = sla.lu_solve(sla.lu_factor(self._mode_matrix(m, kk)), b)
            out[(m, kk)] = (x[:3 * N].reshape(3, N), x[4 * N].real if mean else 0.0)
        return out

    def step(self, U, nsteps=1):
        """Predictor-corrector steps (section 2); returns the new state."""
        p = self.p
        for _ in range(nsteps):
            Nj = self.nonlinear(U)
            Uq, beta_p = self.solve(U, Nj)
            for _q in range(p.n_corr):
                Nq = self.nonlinear(Uq)
                Uq, beta_p = self.solve(U, p.c * Nq + (1.0 - p.c) * Nj)
            U = Uq
            self.beta = beta_p * p.Re / 4.0
        return U

    # ---- diagnostics (section 3.2: E, I, D normalised by laminar values)
    def energy(self, U):
        p = self.p
        wm = np.where(np.arange(p.M) == 0, 1.0, 2.0)
        W = self.curl(U)
        eu = (np.abs(U) ** 2).sum(axis=(0, 2))  # (M, N)
        ew = (np.abs(W) ** 2).sum(axis=(0, 2))
        S_u = float((wm[:, None] * eu).sum(axis=0) @ self.w)
        S_w = float((wm[:, None] * ew).sum(axis=0) @ self.w)
        flux = float(U[2, 0, p.K - 1].real @ self.w)
        E = 6.0 * S_u            # E_lam: int (1-r^2)^2 r dr = 1/6, times 1/2
        I = 4.0 * (1.0 + self.beta) * flux  # I_lam: (4/Re) int (1-r^2) r dr
        D = S_w                  # D_lam: (1/Re) int (2r)^2 r dr = 1/Re
        return np.array([E, I, D])

    def wall_residual(self, U):
        """max |u(1)| and max |div u(1)| over all modes (the vector g)."""
        p, r = self.p, self.r
        g_u = float(np.abs(U[:, :, :, -1]).max())
        div = self.divergence(U)[:, :, -1]
        div[0, p.K - 1] = 0.0  # (0,0) carries the pressure gauge instead
        return g_u, float(np.abs(div).max())

    @staticmethod
    def hermitian_project(U):
        """Impose A(-k, 0) = conj A(k, 0) (real fields)."""
        V = U.copy()
        V[:, 0] = 0.5 * (U[:, 0] + np.conj(U[:, 0, ::-1]))
        return V


def change_resolution(U, N2, K2, M2, m_p):
    """A state (3, M1, 2K1-1, N1) at resolution (N2, K2, M2), same m_p
    (section 2: initial conditions of another resolution are truncated or
    interpolated).  Fourier modes present in both are copied, others zero;
    each radial profile is evaluated at the new points by the Lagrange
    polynomial through the 9 nodes of the parity-extended old mesh nearest to
    the new point (reading R3's extension), its basis written out as
    products."""
    _, M1, nk1, N1 = U.shape
    K1 = (nk1 + 1) // 2
    r1, r2 = mesh(N1), mesh(N2)
    ext = np.concatenate([-r1[::-1], r1])
    out = np.zeros((3, M2, 2 * K2 - 1, N2), dtype=np.complex128)
    for n in range(N2):
        z = r2[n]
        q = int(np.argmin(np.abs(ext - z)))
        f = min(max(q - 4, 0), 2 * N1 - 9)
        nodes = ext[f:f + 9]
        basis = np.array([np.prod([(z - nodes[j]) / (nodes[i] - nodes[j]) for j in range(9) if j != i])
                          for i in range(9)])
        for c in range(3):
            for m in range(min(M1, M2)):
                mt = m_p * m
                parity = (-1) ** mt if c == 2 else (-1) ** (mt + 1)
                for k in range(-(min(K1, K2) - 1), min(K1, K2)):
                    prof = U[c, m, k + K1 - 1]
                    vals = np.array([prof[e - N1] if e >= N1 else parity * prof[N1 - 1 - e]
                                     for e in range(f, f + 9)])
                    out[c, m, k + K2 - 1, n] = basis @ vals
    return out
