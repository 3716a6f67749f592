"""Counter-based random initial data (Sec. 2.2, random initial condition).

The paper draws the initial condition at random but does not name a
generator.  Both sides of every comparison use one counter-based generator,
SplitMix64 as published by Steele, Lea and Flood (OOPSLA 2014), so that the
value drawn for (vertex z, component i) does not depend on the vertex order
or on the device:

    U(z, i) = (splitmix64(seed XOR splitmix64(z*m + i)) >> 11) * 2^-53

Two initial-data kinds are produced:

* uniform: u_i(z) = U(z, i) in [0, 1) for every component;
* one-hot (the paper's choice): one component c(z) = floor(m * U(z, 0)) is
  set to 1 at vertex z and the others to 0.

Normalising each component in L2(Gamma_h) is part of the method and is done
by the consumer, not here.
"""

from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output function applied to the counter x (uint64, wraps mod 2^64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n_vert: int, m: int):
    """U[z, i] in [0, 1), float64, shape (n_vert, m)."""
    z = np.arange(n_vert, dtype=np.uint64)[:, None]
    i = np.arange(m, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        ctr = z * np.uint64(m) + i
    h = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ splitmix64(ctr))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def onehot_choice(seed: int, n_vert: int, m: int):
    """c(z) = floor(m * U(z, 0)) in {0..m-1}, int32, shape (n_vert,)."""
    u0 = uniform01(seed, n_vert, m)[:, 0]
    return np.minimum((u0 * m).astype(np.int64), m - 1).astype(np.int32)


def initial_values(kind: str, seed: int, n_vert: int, m: int):
    """Un-normalised initial values (n_vert, m) float64 for kind 'uniform' or 'onehot'."""
    if kind == "uniform":
        return uniform01(seed, n_vert, m)
    if kind == "onehot":
        c = onehot_choice(seed, n_vert, m)
        u = np.zeros((n_vert, m), dtype=np.float64)
        u[np.arange(n_vert), c] = 1.0
        return u
    raise ValueError(f"unknown initial-data kind {kind!r}")
