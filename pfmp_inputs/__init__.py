"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only draws random numbers (numpy PCG64, so the streams are identical on
x86 and Arm hosts).  It holds none of the method's arithmetic: turning algebra
coefficients into SU(3) links, spinors into pseudofermions, etc. is done separately by
the oracle and by the CUDA library.

Layouts are the canonical host layouts of the C-ABI: lexicographic site index
x + Lx (y + Ly (z + Lz t)), then direction / spin / colour.
"""
import numpy as np


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def volume(dims):
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def gauge_algebra(dims, seed):
    """h[site, mu, a] ~ N(0, 1): coefficients of H = sum_a h_a T_a, one per link."""
    return _rng(seed, 1).standard_normal((volume(dims), 4, 8))


def spinor(dims, seed, n=None):
    """Complex Gaussian spinor field(s) psi[site, spin, colour] with Re, Im ~ N(0, 1/2),
    i.e. density exp(-psi^dag psi).  ``n`` adds a leading batch dimension."""
    shape = (volume(dims), 4, 3) if n is None else (n, volume(dims), 4, 3)
    g = _rng(seed, 2)
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im) * np.sqrt(0.5)


def momenta(dims, seed):
    """p[site, mu, a] ~ N(0, 1): HMC momenta P = sum_a p_a T_a (density exp(-tr P^2))."""
    return _rng(seed, 3).standard_normal((volume(dims), 4, 8))


def uniform(seed, n=1):
    """Uniform numbers in [0, 1) for the Metropolis test."""
    return _rng(seed, 4).random(n)


def uniform_range(seed, lo, hi, n):
    return lo + (hi - lo) * _rng(seed, 5).random(n)


def integers(seed, lo, hi, n):
    return _rng(seed, 6).integers(lo, hi + 1, n)


def nn_weights(channels, seed, scale=0.3):
    """Initial weights of the gauge-covariant network: per layer a complex array
    W[9][c_out][c_in][4][4] of Gaussians scaled by scale / (4 sqrt(9 c_in)), with the
    identity added to the on-site 4x4 block of matching channels (c < min(c_in, c_out))
    so that the untrained network starts near a multiple of the identity map."""
    g = _rng(seed, 7)
    ws = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        w = (g.standard_normal((9, cout, cin, 4, 4)) + 1j * g.standard_normal((9, cout, cin, 4, 4)))
        w *= scale / (4.0 * np.sqrt(9 * cin))
        for c in range(min(cin, cout)):
            w[0, c, c] += np.eye(4)
        ws.append(w)
    return ws
