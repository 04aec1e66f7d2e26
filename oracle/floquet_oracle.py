"""Plain FP64 CPU oracle for the leading eigenvalues of linear maps and the
Floquet multipliers of pipe-flow states.

TEST INFRASTRUCTURE ONLY: imported by tests/ alone; shares no code with the
CUDA library.

  * arnoldi(apply, v0, k): the textbook Arnoldi process -- Krylov basis by
    modified Gram-Schmidt, Hessenberg matrix H -- with the Ritz values taken
    as the eigenvalues of H (numpy.linalg.eigvals as the library step).
  * floquet(oracle, u, T, s, ...): the linearised period map
    dv -> sigma_s DPhi_T(u) dv by a forward difference of two oracle
    integrations, on the independent real coefficients of a state (m = 0
    with k >= 0 and no imaginary part at k = m = 0; all k for m > 0),
    sigma_s the axial shift (mode k times e^{i alpha k s}).
"""
import numpy as np


def arnoldi(apply, v0, k):
    """Ritz values (sorted by decreasing modulus) of k Arnoldi steps."""
    n = v0.size
    V = np.zeros((k + 1, n))
    H = np.zeros((k + 1, k))
    V[0] = v0 / np.linalg.norm(v0)
    for j in range(k):
        w = apply(V[j])
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            k = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    ev = np.linalg.eigvals(H[:k, :k])
    return ev[np.argsort(-np.abs(ev), kind="stable")]


def independent_mask(K, M):
    """Boolean masks (real part, imaginary part) over a state's (m, kk) modes
    marking the independent real coefficients."""
    nk = 2 * K - 1
    k = np.arange(nk) - (K - 1)
    re = np.ones((M, nk), dtype=bool)
    re[0, k < 0] = False
    im = re.copy()
    im[0, K - 1] = False
    return re, im


def pack(U, K, M):
    re, im = independent_mask(K, M)
    return np.concatenate([U.real[:, re].ravel(), U.imag[:, im].ravel()])


def unpack(x, K, M, N):
    re, im = independent_mask(K, M)
    nre = 3 * int(re.sum()) * N
    U = np.zeros((3, M, 2 * K - 1, N), dtype=np.complex128)
    U.real[:, re] = x[:nre].reshape(3, -1, N)
    U.imag[:, im] = x[nre:].reshape(3, -1, N)
    # m = 0, k < 0 from the conjugate symmetry of a real field
    nk = 2 * K - 1
    for kk in range(K - 1):
        U[:, 0, kk] = np.conj(U[:, 0, nk - 1 - kk])
    return U


def shifted(U, s, alpha, K):
    k = np.arange(2 * K - 1) - (K - 1)
    return U * np.exp(1j * alpha * k * s)[None, None, :, None]


def floquet(oracle, U, T, s, v0, k, eps=1e-7):
    """Leading Floquet multipliers of state U: period T = nsteps * oracle dt."""
    p = oracle.p
    nsteps = int(round(T / p.dt))
    base = pack(shifted(oracle.step(U, nsteps), s, p.alpha, p.K), p.K, p.M)
    u = pack(U, p.K, p.M)

    def apply(v):
        e = eps * np.linalg.norm(u) / np.linalg.norm(v)
        W = oracle.step(unpack(u + e * v, p.K, p.M, p.N), nsteps)
        return (pack(shifted(W, s, p.alpha, p.K), p.K, p.M) - base) / e

    return arnoldi(apply, v0, k)
