"""Pins for the shared seeded input generators (meshes and random initial data)."""

import numpy as np
import pytest

import workload as w


def _edges(tri):
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 0)
    return e


def _closed_oriented(tri):
    """Every directed edge appears once and its reverse once (closed, consistently oriented)."""
    e = _edges(tri).astype(np.int64)
    n = int(tri.max()) + 1
    fwd = e[:, 0] * n + e[:, 1]
    rev = e[:, 1] * n + e[:, 0]
    return len(np.unique(fwd)) == len(fwd) and np.array_equal(np.sort(fwd), np.sort(rev))


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_counts_and_surface(level):
    xyz, tri = w.icosphere(level)
    assert xyz.shape == (10 * 4 ** level + 2, 3)
    assert tri.shape == (20 * 4 ** level, 3)
    assert np.abs(np.linalg.norm(xyz, axis=1) - 1).max() < 1e-15
    assert _closed_oriented(tri)
    n_e = len(_edges(tri)) // 2
    assert xyz.shape[0] - n_e + tri.shape[0] == 2  # Euler characteristic of the sphere
    # outward orientation: signed volume positive
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    assert (np.einsum("fk,fk->f", np.cross(b - a, c - a), a + b + c) > 0).all()
    # no duplicate vertices
    assert len(np.unique(np.round(xyz, 12), axis=0)) == xyz.shape[0]


def test_icosphere_level_counts_of_the_workloads():
    # the level-8 sphere of the headline workload has 655 362 vertices
    for level, n in [(4, 2562), (7, 163842), (8, 655362)]:
        assert 10 * 4 ** level + 2 == n
    xyz, tri = w.icosphere(7)
    assert xyz.shape[0] == 163842 and tri.shape[0] == 327680


def test_torus_surface_and_topology():
    R, r = 1.0, 0.4
    xyz, tri = w.torus(16, 8, R, r)
    assert xyz.shape == (128, 3) and tri.shape == (256, 3)
    rho = np.hypot(xyz[:, 0], xyz[:, 1])
    assert np.abs((rho - R) ** 2 + xyz[:, 2] ** 2 - r * r).max() < 1e-14
    assert _closed_oriented(tri)
    n_e = len(_edges(tri)) // 2
    assert xyz.shape[0] - n_e + tri.shape[0] == 0  # genus one
    # outward normals: normal points away from the tube centre circle
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    cen = (a + b + c) / 3
    ring = cen.copy()
    ring[:, 2] = 0
    ring *= R / np.linalg.norm(ring, axis=1, keepdims=True)
    assert (np.einsum("fk,fk->f", np.cross(b - a, c - a), cen - ring) > 0).all()


def test_ellipsoid_surface():
    xyz, tri = w.ellipsoid(3, 1.0, 0.8, 0.6)
    q = (xyz[:, 0] / 1.0) ** 2 + (xyz[:, 1] / 0.8) ** 2 + (xyz[:, 2] / 0.6) ** 2
    assert np.abs(q - 1).max() < 1e-14
    sx, st = w.icosphere(3)
    assert np.array_equal(tri, st)
    # radial map: same direction as the sphere vertex
    assert np.abs(np.cross(xyz, sx)).max() < 1e-15


def test_splitmix64_published_outputs():
    # First two outputs of SplitMix64 started from state 0 (Steele, Lea, Flood 2014)
    assert int(w.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    assert int(w.splitmix64(np.uint64(0x9E3779B97F4A7C15))) == 0x6E789E6AA1B965F4


def test_uniform_is_counter_based_and_in_range():
    U = w.uniform01(1234, 50, 3)
    assert U.min() >= 0 and U.max() < 1
    # value at (z, i) depends only on (seed, z*m + i)
    U2 = w.uniform01(1234, 80, 3)
    assert np.array_equal(U, U2[:50])
    assert not np.array_equal(U, w.uniform01(1235, 50, 3))
    # mean / variance of U(0,1) on a larger draw
    V = w.uniform01(7, 20000, 4)
    assert abs(V.mean() - 0.5) < 0.01 and abs(V.var() - 1 / 12) < 0.005


def test_onehot_choice():
    m = 5
    c = w.onehot_choice(3, 10000, m)
    assert c.min() == 0 and c.max() == m - 1
    counts = np.bincount(c, minlength=m)
    assert (np.abs(counts / 10000 - 1 / m) < 0.02).all()
    u = w.initial_values("onehot", 3, 10000, m)
    assert np.array_equal(u.sum(1), np.ones(10000))
    assert np.array_equal(u.argmax(1), c)
