"""Seeded synthetic inputs shared by the GPU path, the oracle and the tests.

This module only draws and lays out inputs; it holds none of the method's
arithmetic (no forces, correlators or integrals).  Random numbers come from
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), turned into normal deviates by the Box-Muller
transform (Box and Muller, 1958).  Both are implemented here from their
published definitions so that every machine draws the same numbers.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs for the given 64-bit seed."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def fcc_lattice(cells: int, rho: float):
    """Positions [3, 4*cells^3] of an fcc crystal of number density rho in a
    periodic cubic box, shifted by a quarter lattice spacing so that no atom
    sits on a box face; returns (r, L)."""
    a = (4.0 / rho) ** (1.0 / 3.0)
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(cells, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    origins = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    pos = (origins[:, None, :] + basis[None, :, :] + 0.25).reshape(-1, 3) * a
    return np.ascontiguousarray(pos.T), cells * a


def maxwell_velocities(n: int, T: float, seed: int, masses_of=None):
    """Velocities [3, n] drawn from Maxwell-Boltzmann at temperature T
    (kB = 1), with the centre-of-mass momentum removed and then rescaled so
    that the instantaneous temperature with 3n - 3 degrees of freedom is
    exactly T."""
    m = np.ones(n) if masses_of is None else np.asarray(masses_of, dtype=np.float64)
    v = normal(seed, 3 * n).reshape(3, n) * np.sqrt(T / m)[None, :]
    p = (v * m[None, :]).sum(axis=1) / m.sum()
    v -= p[:, None]
    t_now = (m[None, :] * v * v).sum() / (3.0 * n - 3.0)
    v *= math.sqrt(T / t_now)
    return np.ascontiguousarray(v)


def lj_system(cells: int, rho: float = 0.8442, T: float = 0.722, seed: int = 1):
    """A one-species LJ system: fcc start at density rho, Maxwell-Boltzmann
    velocities at T.  Returns dict(r, v, L, n, types, masses)."""
    r, L = fcc_lattice(cells, rho)
    n = r.shape[1]
    v = maxwell_velocities(n, T, seed)
    return dict(r=r, v=v, L=L, n=n, types=np.zeros(n, dtype=np.int32), masses=np.array([1.0]))


def cells_for_atoms(n_target: int, lo: int = 5, hi: int = 20) -> int:
    """fcc cells per side k with 4 k^3 closest to n_target, k in [lo, hi]."""
    k = int(round((n_target / 4.0) ** (1.0 / 3.0)))
    return max(lo, min(hi, k))


def ar1_series(nseries: int, S: int, phi: float, seed: int) -> np.ndarray:
    """nseries stationary AR(1) series x_t = phi x_{t-1} + sqrt(1-phi^2) e_t
    of length S with unit variance, shape [S, nseries] (one row per time)."""
    e = normal(seed, S * nseries).reshape(S, nseries)
    x = np.empty((S, nseries))
    x[0] = e[0]
    c = math.sqrt(1.0 - phi * phi)
    for t in range(1, S):
        x[t] = phi * x[t - 1] + c * e[t]
    return x


def mlp_init(seed: int, dims, bias_scale: float = 0.0):
    """Weights of a fully connected network with layer widths dims
    (n_in, hidden..., n_out): Glorot-uniform matrices W [out, in] with
    limit sqrt(6 / (in + out)) (Glorot and Bengio, 2010) and biases uniform
    in [-bias_scale, bias_scale].  Returns [(W, b)] per layer."""
    out = []
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        lim = math.sqrt(6.0 / (fi + fo))
        W = (2.0 * uniform01(seed * 1000 + 2 * l, fo * fi) - 1.0).reshape(fo, fi) * lim
        b = (2.0 * uniform01(seed * 1000 + 2 * l + 1, fo) - 1.0) * bias_scale
        out.append((W, b))
    return out


def permutations(seed: int, count: int, n: int) -> np.ndarray:
    """count independent uniform permutations of range(n), shape [count, n],
    by sorting SplitMix64 keys (ties broken by index)."""
    keys = splitmix64(seed, count * n).reshape(count, n)
    return np.argsort(keys, axis=1, kind="stable").astype(np.int64)


def rock_salt_lattice(cells: int, rho: float):
    """Ions of a rock-salt crystal of number density rho (cells^3 cubic
    unit cells of 8 ions) in a periodic cubic box, shifted by a quarter
    spacing: positions [3, n] (cations first, then anions), types (0 for
    cations, 1 for anions) and the box side."""
    a = (8.0 / rho) ** (1.0 / 3.0)
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(cells, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    org = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    cat = (org[:, None, :] + base[None] + 0.25).reshape(-1, 3)
    an = (org[:, None, :] + base[None] + np.array([0.75, 0.25, 0.25])).reshape(-1, 3)
    pos = np.concatenate([cat, an]) * a
    types = np.concatenate([np.zeros(len(cat), dtype=np.int32), np.ones(len(an), dtype=np.int32)])
    return np.ascontiguousarray(pos.T), types, cells * a


def ionic_system(cells: int, rho: float, T: float, seed: int, masses=(22.99, 35.45), jitter: float = 0.0):
    """A binary ionic melt start: a rock-salt lattice of number density rho
    with every ion displaced uniformly by up to +-jitter per axis, and
    Maxwell-Boltzmann velocities at temperature T (kB = 1, in the caller's
    energy unit) for the two masses.  Returns dict(r, v, types, L, n, masses)."""
    r, types, L = rock_salt_lattice(cells, rho)
    n = r.shape[1]
    if jitter:
        r = r + jitter * (2.0 * uniform01(seed + 77, 3 * n).reshape(3, n) - 1.0)
    m = np.asarray(masses, dtype=np.float64)[types]
    v = maxwell_velocities(n, T, seed, masses_of=m)
    return dict(r=np.ascontiguousarray(r), v=v, types=types, L=L, n=n, masses=np.asarray(masses, dtype=np.float64))
