"""Seeded synthetic pipe-flow states (the only module shared by the CUDA path's
tests/benchmark and the CPU oracle).

It holds the input recipe only -- random draws and analytic, divergence-free
polynomial profiles sampled on the radial points -- and none of the time-step
arithmetic.  States use the library's host layout: complex128 array of shape
(3, M, 2K-1, N) holding (u_r, u_theta, u_z) of the TOTAL velocity, axial index
kk = k + K - 1, radial index n ascending (r_N = 1 is the wall).

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) as a counter stream,
Box-Muller for normal deviates.  The perturbation recipe per Fourier mode
(k, m), with m~ = m_p*m and s(r) = (1 - r^2)^2:
  k != 0        : u+ = a r^(m~+1) s, u- = b r^|m~-1| s, u_z from div u = 0
  k == 0, m != 0: streamfunction psi = c r^m~ s, u_r = i m~ psi / r,
                  u_theta = -psi', plus u_z = d r^m~ (1 - r^2)
  k == 0, m == 0: u_theta = e r (1 - r^2), u_z = f (1 - r^2)(1 - 3 r^2)
each mode weighted by a spectral envelope, then the whole perturbation scaled
so its volume rms equals the requested amplitude; Hagen-Poiseuille 1 - r^2 is
added to the (0,0) axial mode.  These profiles vanish at the wall.
"""
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count):
    """`count` consecutive SplitMix64 outputs for `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed, count):
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def complex_normals(seed, count):
    """`count` complex deviates, real and imaginary parts each N(0, 1)."""
    u = uniforms(seed, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * np.pi * u2) + 1j * rad * np.sin(2.0 * np.pi * u2)


def radial_points(N):
    """Radial points r_n = cos(pi (N - n) / (2N - 1)), n = 1..N (r_N = 1)."""
    n = np.arange(1, N + 1, dtype=np.float64)
    return np.cos(np.pi * (N - n) / (2 * N - 1))


def _volume_rms(U, r):
    """Volume rms of a spectral field by the trapezoid rule in r (input scaling only)."""
    M = U.shape[1]
    wm = np.where(np.arange(M) == 0, 1.0, 2.0)
    e = (np.abs(U) ** 2).sum(axis=(0, 2))  # (M, N)
    e = (wm[:, None] * e).sum(axis=0)  # (N,)
    rr = np.concatenate([[0.0], r])
    f = np.concatenate([[0.0], e * r])
    integral = np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(rr))
    return math.sqrt(2.0 * integral)  # divide by int_0^1 r dr = 1/2


def envelope_exp(k, m, K, M):
    """exp(-|k| - m): the small plain-method workload's spectral envelope."""
    return math.exp(-abs(k) - m)


def envelope_puff(k, m, K, M):
    """exp(-m) times the spectrum of a Gaussian of width L_z/4 in z."""
    return math.exp(-m) * math.exp(-(math.pi ** 2) * k * k / 8.0)


def envelope_broadband(k, m, K, M):
    """exp(-3(|k|/K + m/M)): broadband turbulent-start envelope."""
    return math.exp(-3.0 * (abs(k) / K + m / M))


def seeded_state(N, K, M, m_p, alpha, amplitude, seed, envelope=envelope_exp,
                 laminar=True, r=None):
    """Total-velocity state (3, M, 2K-1, N) complex128 following the recipe
    above, sampled at the radial points r (default: radial_points(N))."""
    r = radial_points(N) if r is None else np.asarray(r, dtype=np.float64)
    nk = 2 * K - 1
    s = (1.0 - r * r) ** 2
    ds = -4.0 * r * (1.0 - r * r)
    draws = complex_normals(seed, 6 * nk * M)
    U = np.zeros((3, M, nk, N), dtype=np.complex128)
    for m in range(M):
        mt = m_p * m
        for kk in range(nk):
            k = kk - (K - 1)
            if m == 0 and k < 0:
                continue  # filled by Hermitian symmetry below
            a, b, c, d, e, f = draws[6 * (m * nk + kk): 6 * (m * nk + kk) + 6]
            w = envelope(k, m, K, M)
            if k != 0:
                q = abs(mt - 1)
                up = a * r ** (mt + 1) * s
                um = b * r ** q * s
                pp = a * ((2 * mt + 2) * r ** (mt + 1) * s + r ** (mt + 2) * ds)
                pm = b * ((q + 1 - mt) * r ** q * s + r ** (q + 1) * ds)
                uz = 1j / (2.0 * alpha * k * r) * (pp + pm)
                ur = 0.5 * (up + um)
                ut = (up - um) / 2j
            elif m != 0:
                psi = c * r ** mt * s
                dpsi = c * (mt * r ** (mt - 1) * s + r ** mt * ds)
                ur = 1j * mt * psi / r
                ut = -dpsi
                uz = d * r ** mt * (1.0 - r * r)
            else:
                ur = np.zeros(N)
                ut = e.real * r * (1.0 - r * r)
                uz = f.real * (1.0 - r * r) * (1.0 - 3.0 * r * r)
            U[0, m, kk] = w * ur
            U[1, m, kk] = w * ut
            U[2, m, kk] = w * uz
    for kk in range(K, nk):  # m = 0, k > 0  ->  k < 0 by conjugation
        U[:, 0, nk - 1 - kk] = np.conj(U[:, 0, kk])
    rms = _volume_rms(U, r)
    if rms > 0:
        U *= amplitude / rms
    if laminar:
        U[2, 0, K - 1] += 1.0 - r * r
    return U


def laminar_state(N, K, M, r=None):
    """Hagen-Poiseuille flow u_z = 1 - r^2 in the host layout (at the points r,
    default radial_points(N))."""
    r = radial_points(N) if r is None else np.asarray(r, dtype=np.float64)
    U = np.zeros((3, M, 2 * K - 1, N), dtype=np.complex128)
    U[2, 0, K - 1] = 1.0 - r * r
    return U


# Named workloads: (N, K, M, m_p, alpha, Re, dt, amplitude, seed, envelope)
WORKLOADS = {
    "small": dict(N=32, K=16, M=16, m_p=1, alpha=1.25, Re=2000.0, dt=0.01,
                  amplitude=1e-2, seed=1705038381, envelope=envelope_exp),
    "medium": dict(N=48, K=32, M=24, m_p=2, alpha=1.25, Re=2400.0, dt=0.005,
                   amplitude=0.1, seed=1705038382, envelope=envelope_puff),
    "large": dict(N=128, K=128, M=128, m_p=1, alpha=0.4, Re=5300.0, dt=0.002,
                  amplitude=0.3, seed=1705038384, envelope=envelope_broadband),
}


def stretched_mesh(N, beta=1.8):
    """A radial mesh other than the default one, for testing user meshes:
    r_n = sinh(beta x_n) / sinh(beta), x_n = n / N (n = 1..N), clustered
    towards the axis instead of the wall (r_N = 1)."""
    x = np.arange(1, N + 1, dtype=np.float64) / N
    r = np.sinh(beta * x) / math.sinh(beta)
    r[-1] = 1.0
    return r


def workload_state(name):
    w = WORKLOADS[name]
    return seeded_state(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["amplitude"],
                        w["seed"], w["envelope"])
