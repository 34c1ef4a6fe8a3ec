"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

This module holds no arithmetic of the method: it only draws seeded random
arrays (numpy's PCG64) shaped like the paper's workloads -- a homogeneous
field value plus small fluctuations, random link angles, random electric
fields -- that both sides then receive as the same input.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(int(seed))


def scalar_state(N, nf=1, seed=0, fbar=(1.0, 0.0), amp=1e-2, pamp=1e-2, pbar=(0.0, 0.0)):
    """Homogeneous values plus white-noise fluctuations of relative size amp."""
    g = rng(seed)
    phi = np.empty((nf, N, N, N))
    pi = np.empty((nf, N, N, N))
    for f in range(nf):
        phi[f] = fbar[f] + amp * g.standard_normal((N, N, N))
        pi[f] = pbar[f] + pamp * g.standard_normal((N, N, N))
    return phi, pi


def plane_wave(N, m, amp=1.0, phase=0.0):
    """cos(2 pi m.n / N + phase) on an N^3 lattice, indexed [z, y, x]."""
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    arg = 2.0 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / N + phase
    return amp * np.cos(arg)


def gauge_state(N, seed=0, theta_amp=1e-1, e_amp=1e-1):
    """Random link angles theta_i and electric fields E_i, shape (3, N, N, N)."""
    g = rng(seed)
    return theta_amp * g.standard_normal((3, N, N, N)), e_amp * g.standard_normal((3, N, N, N))


def solenoidal_field(N, seed=0, amp=1e-1, dtype=np.float64):
    """Random link field E_i(n) with zero backward-difference divergence on the periodic
    lattice: E = curl- v (E_i = [v_k(n) - v_k(n - e_j)] - [v_j(n) - v_j(n - e_k)], (i, j, k)
    cyclic, direction 0 the fastest index) of a white-noise v, scaled to rms amp."""
    v = rng(seed).standard_normal((3, N, N, N)).astype(dtype)

    def back(f, d):  # f(n) - f(n - e_d)
        return f - np.roll(f, 1, axis=2 - d)

    E = np.stack([back(v[(i + 2) % 3], (i + 1) % 3) - back(v[(i + 1) % 3], (i + 2) % 3) for i in range(3)])
    return (amp / max(float(np.sqrt(np.mean(E * E))), 1e-300)) * E
