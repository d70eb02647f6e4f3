"""Seeded synthetic moonlet disks (input generation only).

This module draws the initial conditions that both the CUDA path and the
CPU oracle consume.  It holds none of the falcON step's arithmetic: it only
turns a seed into positions, velocities, masses and radii shaped like the
disks of the paper's performance runs (Sect. 4.2: moonlets orbiting a central
mass with small eccentricities and inclinations, elastic radii spread).

Recipe (units G = M_c = R_c = 1):
  * semi-major axis a ~ U[a_lo, a_hi]            (default [2, 10])
  * eccentricity e ~ Rayleigh(sigma_e)            (default 0.05)
  * inclination i ~ Rayleigh(sigma_i) [rad]       (default 0.025)
  * mean anomaly, argument of pericentre, node ~ U[0, 2 pi)
  * radius R from dN/dR ~ R^-3.5 on [R_lo, R_hi]  (default [1e-3, 1e-2]),
    drawn by inverse CDF
  * mass m ~ R^3 (uniform density) scaled so that sum(m) = disk_mass (0.02)
  * Kepler's equation solved by Newton iteration to |dE| < 1e-15, then the
    usual rotation by (omega, i, Omega) with mu = G * M_c.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used
as a counter-based stream: the k-th output for a seed is
mix(seed + (k + 1) * 0x9E3779B97F4A7C15).  Particle i consumes draws
7 i + 0 .. 7 i + 6 in the order (a, e, i, M, omega, Omega, R).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream for `seed`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _solve_kepler(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    E = M + e * np.sin(M)
    for _ in range(60):
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = E - dE
        if np.all(np.abs(dE) < 1e-15):
            break
    return E


def make_disk(n: int, seed: int, *, a_lo=2.0, a_hi=10.0, sigma_e=0.05, sigma_i=0.025,
              r_lo=1e-3, r_hi=1e-2, disk_mass=0.02, G=1.0, central_mass=1.0):
    """Return dict(pos[n,3], vel[n,3], mass[n], radius[n]) as float64 arrays."""
    n = int(n)
    u = uniforms(seed, 7 * n).reshape(n, 7) if n > 0 else np.zeros((0, 7))
    a = a_lo + (a_hi - a_lo) * u[:, 0]
    e = sigma_e * np.sqrt(-2.0 * np.log1p(-u[:, 1]))
    inc = sigma_i * np.sqrt(-2.0 * np.log1p(-u[:, 2]))
    e = np.minimum(e, 0.9)  # Rayleigh tail beyond 0.9 has probability exp(-162)
    two_pi = 2.0 * np.pi
    M, om, Om = two_pi * u[:, 3], two_pi * u[:, 4], two_pi * u[:, 5]
    lo, hi = r_lo ** -2.5, r_hi ** -2.5
    R = (lo + u[:, 6] * (hi - lo)) ** (-1.0 / 2.5)
    m = R ** 3
    m *= disk_mass / m.sum() if n > 0 else 1.0

    mu = G * central_mass
    E = _solve_kepler(M, e)
    cE, sE = np.cos(E), np.sin(E)
    sq = np.sqrt(1.0 - e * e)
    xp, yp = a * (cE - e), a * sq * sE
    Edot = np.sqrt(mu / a ** 3) / (1.0 - e * cE)
    vxp, vyp = -a * sE * Edot, a * sq * cE * Edot
    cO, sO, co, so, ci, si = np.cos(Om), np.sin(Om), np.cos(om), np.sin(om), np.cos(inc), np.sin(inc)
    r11, r12 = cO * co - sO * so * ci, -cO * so - sO * co * ci
    r21, r22 = sO * co + cO * so * ci, -sO * so + cO * co * ci
    r31, r32 = so * si, co * si
    pos = np.stack([r11 * xp + r12 * yp, r21 * xp + r22 * yp, r31 * xp + r32 * yp], axis=1)
    vel = np.stack([r11 * vxp + r12 * vyp, r21 * vxp + r22 * vyp, r31 * vxp + r32 * vyp], axis=1)
    return {"pos": np.ascontiguousarray(pos), "vel": np.ascontiguousarray(vel),
            "mass": np.ascontiguousarray(m), "radius": np.ascontiguousarray(R)}


def subsample(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct particle indices in [0, n), drawn from the seed (sorted)."""
    k = min(int(k), int(n))
    keys = splitmix64(seed ^ 0x5EED5EED, n)
    return np.sort(np.argsort(keys, kind="stable")[:k]).astype(np.int64)


def ensemble_sizes(n_disks: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Disk sizes log-uniform in [lo, hi] (integers), one per disk."""
    u = uniforms(seed ^ 0xD15C5, n_disks)
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
