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


# --- refinement with projection, surface (D) (Sec. 3.3, Sec. 3.4) ----------


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_refining_the_icosphere_gives_the_next_level(level):
    x, t = w.icosphere(level)
    xf, tf, par = w.refine(x, t, ("sphere",))
    x1, t1 = w.icosphere(level + 1)
    assert np.array_equal(xf, x1) and np.array_equal(tf, t1)
    assert np.array_equal(par[: len(x)], np.stack([np.arange(len(x))] * 2, 1))


def test_flat_refinement_midpoints_and_children():
    x, t = w.torus(6, 5, 1.0, 0.4)
    xf, tf, par = w.refine(x, t, ("none",))
    n, f = len(x), len(t)
    assert len(xf) == n + 3 * f // 2 and len(tf) == 4 * f  # closed surface: E = 3F/2
    assert np.array_equal(xf[n:], 0.5 * (x[par[n:, 0]] + x[par[n:, 1]]))
    assert (par[n:, 0] < par[n:, 1]).all()
    # the four children of a triangle tile it: equal total area, shared corners
    def area(p, tri):
        return 0.5 * np.linalg.norm(np.cross(p[tri[:, 1]] - p[tri[:, 0]], p[tri[:, 2]] - p[tri[:, 0]]), axis=1)
    a0 = area(x, t)
    a1 = area(xf, tf).reshape(4, f).sum(0)
    assert np.allclose(a0, a1, rtol=1e-13)
    assert np.array_equal(tf[:f, 0], t[:, 0]) and np.array_equal(tf[f:2 * f, 0], t[:, 1])
    # every edge of the fine mesh is shared by exactly two triangles
    e = np.sort(np.concatenate([tf[:, [0, 1]], tf[:, [1, 2]], tf[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert (cnt == 2).all()


def test_refinement_projects_onto_torus_and_ellipsoid():
    x, t = w.torus(12, 8, 1.0, 0.4)
    xf, _, _ = w.refine(x, t, ("torus", 1.0, 0.4))
    rho = np.sqrt(xf[:, 0] ** 2 + xf[:, 1] ** 2)
    assert np.abs((rho - 1.0) ** 2 + xf[:, 2] ** 2 - 0.16).max() < 1e-14
    x, t = w.ellipsoid(2, 1.0, 0.8, 0.6)
    xf, _, _ = w.refine(x, t, ("ellipsoid", 1.0, 0.8, 0.6))
    q = (xf[:, 0] / 1.0) ** 2 + (xf[:, 1] / 0.8) ** 2 + (xf[:, 2] / 0.6) ** 2
    assert np.abs(q - 1.0).max() < 1e-14


def test_dziuk_surface_mesh():
    for level in range(4):
        x, t = w.dziuk(level)
        assert len(x) == 10 * 4 ** level + 2 and len(t) == 20 * 4 ** level
        phi, grad = w.dziuk_phi(x)
        assert np.abs(phi).max() <= 1e-14
    # outward orientation kept: normals point away from the origin-star
    nrm = np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]])
    assert (np.einsum("ij,ij->i", nrm, x[t].mean(1)) > 0).all()
    # Newton projection of a point already on the surface is the identity;
    # the unit circle x3 = 0 lies on (D)
    s = np.array([[np.cos(0.3), np.sin(0.3), 0.0]])
    assert np.array_equal(w.project_dziuk(s), s)
    # the gradient formula matches central differences
    p = np.array([[0.3, -0.4, 0.5]])
    _, g = w.dziuk_phi(p)
    h = 1e-6
    fd = [(w.dziuk_phi(p + h * e)[0] - w.dziuk_phi(p - h * e)[0])[0] / (2 * h) for e in np.eye(3)]
    assert np.allclose(g[0], fd, atol=1e-8)
