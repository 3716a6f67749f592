"""Triangulated surfaces Gamma_h whose vertices lie on the smooth surface.

Sec. 2.1 asks for a shape-regular triangulation that interpolates Gamma (all
vertices on Gamma).  The generators below produce the three surface families
used by the workloads:

* ``icosphere(level)``: the regular icosahedron, split ``level`` times
  (each triangle into four through its edge midpoints), every new vertex
  projected radially onto the unit sphere.  N = 10*4^L + 2, F = 20*4^L.
* ``ellipsoid(level, a, b, c)``: the icosphere mapped radially onto
  x^2/a^2 + y^2/b^2 + z^2/c^2 = 1.
* ``torus(nu, nv, R, r)``: a structured (u, v) grid on the torus with tube
  radius r around a circle of radius R, each grid quad split along one fixed
  diagonal.

* ``dziuk(level)``: surface (D) of Sec. 3.4, {Phi = 0} with
  Phi(x) = (x1 - x3^2)^2 + x2^2 + x3^2 - 1: the icosahedron's vertices moved
  onto it by Newton projection, then ``level`` refinements whose new vertices
  are projected the same way.
* ``refine(xyz, tri, surface)``: one global refinement (every triangle into
  four through its edge midpoints), each midpoint projected onto the named
  surface; returns the parent edge of every fine vertex as well.

All triangles are oriented with outward normals.  Vertex numbering is
deterministic: the 12 icosahedron vertices first, then at each level the new
midpoint vertices in increasing (min endpoint, max endpoint) order.
"""

from __future__ import annotations

import numpy as np


def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts.append((0.0, s1, s2 * phi))
            pts.append((s1, s2 * phi, 0.0))
            pts.append((s2 * phi, 0.0, s1))
    xyz = np.array(pts, dtype=np.float64)
    # faces = triples of mutually nearest vertices (edge length 2)
    d2 = ((xyz[:, None, :] - xyz[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - 4.0) < 1e-9
    faces = []
    n = len(xyz)
    for a in range(n):
        for b in range(a + 1, n):
            if not adj[a, b]:
                continue
            for c in range(b + 1, n):
                if adj[a, c] and adj[b, c]:
                    nrm = np.cross(xyz[b] - xyz[a], xyz[c] - xyz[a])
                    if np.dot(nrm, xyz[a] + xyz[b] + xyz[c]) > 0:
                        faces.append((a, b, c))
                    else:
                        faces.append((a, c, b))
    tri = np.array(faces, dtype=np.int32)
    assert tri.shape == (20, 3)
    xyz /= np.linalg.norm(xyz, axis=1, keepdims=True)
    return xyz, tri


def _split_once(xyz, tri):
    n = xyz.shape[0]
    a, b, c = tri[:, 0].astype(np.int64), tri[:, 1].astype(np.int64), tri[:, 2].astype(np.int64)
    e = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 0)  # 3 x F x 2
    lo = e.min(axis=2)
    hi = e.max(axis=2)
    key = lo * n + hi
    ukey, inv = np.unique(key.ravel(), return_inverse=True)
    inv = inv.reshape(3, -1)
    ulo = ukey // n
    uhi = ukey % n
    mid = xyz[ulo] + xyz[uhi]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    new_xyz = np.concatenate([xyz, mid], 0)
    ab, bc, ca = n + inv[0], n + inv[1], n + inv[2]
    new_tri = np.concatenate(
        [
            np.stack([a, ab, ca], 1),
            np.stack([b, bc, ab], 1),
            np.stack([c, ca, bc], 1),
            np.stack([ab, bc, ca], 1),
        ],
        0,
    )
    return new_xyz, new_tri.astype(np.int32)


def _project(p, surface):
    """Move the points p[k, 3] onto a surface given as a tuple
    ("none",) | ("sphere",) | ("ellipsoid", a, b, c) | ("torus", R, r) | ("dziuk",)."""
    kind = surface[0]
    if kind == "none":
        return p
    if kind == "sphere":
        return p / np.sqrt(p[:, 0] * p[:, 0] + p[:, 1] * p[:, 1] + p[:, 2] * p[:, 2])[:, None]
    if kind == "ellipsoid":
        a, b, c = surface[1:4]
        q = np.sqrt((p[:, 0] / a) ** 2 + (p[:, 1] / b) ** 2 + (p[:, 2] / c) ** 2)
        return p / q[:, None]
    if kind == "torus":
        R, r = surface[1:3]
        rho = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2)
        ctr = np.stack([R * p[:, 0] / rho, R * p[:, 1] / rho, np.zeros_like(rho)], 1)
        d = p - ctr
        return ctr + r * d / np.linalg.norm(d, axis=1)[:, None]
    if kind == "dziuk":
        return project_dziuk(p)
    raise ValueError(f"unknown surface {surface!r}")


def dziuk_phi(x):
    """Phi of surface (D) and its gradient at the points x[k, 3]."""
    w = x[:, 0] - x[:, 2] ** 2
    phi = w * w + x[:, 1] ** 2 + x[:, 2] ** 2 - 1.0
    grad = np.stack([2.0 * w, 2.0 * x[:, 1], 2.0 * x[:, 2] - 4.0 * x[:, 2] * w], 1)
    return phi, grad


def project_dziuk(x, tol=1e-14, maxit=50):
    """Newton projection onto {Phi = 0}: x <- x - Phi grad / |grad|^2 until
    |Phi| <= tol (at most maxit iterations per point)."""
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(maxit):
        phi, g = dziuk_phi(x)
        act = np.abs(phi) > tol
        if not act.any():
            break
        g2 = (g * g).sum(1)
        x[act] -= (phi[act] / g2[act])[:, None] * g[act]
    return x


def refine(xyz, tri, surface):
    """One global refinement with projection onto `surface`.

    Returns (xyz_fine, tri_fine, parents[N_fine, 2]): the coarse vertices keep
    their numbers (parents (z, z)), the midpoint of edge (lo, hi) becomes
    vertex N + (rank of the edge in (lo, hi) order) with parents (lo, hi); the
    children of triangle t are t, F + t, 2F + t (at its corners a, b, c) and
    3F + t (the middle one).
    """
    n = xyz.shape[0]
    a, b, c = tri[:, 0].astype(np.int64), tri[:, 1].astype(np.int64), tri[:, 2].astype(np.int64)
    e = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 0)
    lo = e.min(axis=2)
    hi = e.max(axis=2)
    ukey, inv = np.unique((lo * n + hi).ravel(), return_inverse=True)
    inv = inv.reshape(3, -1)
    ulo, uhi = ukey // n, ukey % n
    mid = _project(0.5 * (xyz[ulo] + xyz[uhi]), surface)
    ab, bc, ca = n + inv[0], n + inv[1], n + inv[2]
    new_tri = np.concatenate(
        [np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1), np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], 0)
    parents = np.concatenate([np.stack([np.arange(n), np.arange(n)], 1), np.stack([ulo, uhi], 1)], 0)
    return np.concatenate([xyz, mid], 0), new_tri.astype(np.int32), parents.astype(np.int32)


def dziuk(level: int):
    """Surface (D): projected icosahedron refined `level` times (Newton projection)."""
    if level < 0:
        raise ValueError("level must be >= 0")
    xyz, tri = _icosahedron()
    xyz = project_dziuk(xyz)
    for _ in range(level):
        xyz, tri, _ = refine(xyz, tri, ("dziuk",))
    return xyz, tri


def icosphere(level: int):
    """Unit sphere mesh: (xyz[N,3] float64, tri[F,3] int32)."""
    if level < 0:
        raise ValueError("level must be >= 0")
    xyz, tri = _icosahedron()
    for _ in range(level):
        xyz, tri = _split_once(xyz, tri)
    return xyz, tri


def ellipsoid(level: int, a: float, b: float, c: float):
    """Icosphere of the given level mapped radially onto the ellipsoid."""
    xyz, tri = icosphere(level)
    s = np.sqrt((xyz[:, 0] / a) ** 2 + (xyz[:, 1] / b) ** 2 + (xyz[:, 2] / c) ** 2)
    return xyz / s[:, None], tri


def torus(nu: int, nv: int, R: float, r: float):
    """Torus ((R + r cos v) cos u, (R + r cos v) sin u, r sin v) on an nu x nv grid."""
    if nu < 3 or nv < 3:
        raise ValueError("torus grid needs nu, nv >= 3")
    j = np.arange(nu)
    k = np.arange(nv)
    u = 2.0 * np.pi * j / nu
    v = 2.0 * np.pi * k / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    rho = R + r * np.cos(V)
    xyz = np.stack([rho * np.cos(U), rho * np.sin(U), r * np.sin(V)], -1).reshape(-1, 3)
    J, K = np.meshgrid(j, k, indexing="ij")
    J1 = (J + 1) % nu
    K1 = (K + 1) % nv
    v00 = (J * nv + K).ravel()
    v10 = (J1 * nv + K).ravel()
    v11 = (J1 * nv + K1).ravel()
    v01 = (J * nv + K1).ravel()
    tri = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    return xyz.astype(np.float64), tri.astype(np.int32)


def mesh_by_name(spec: str):
    """'sphere:L', 'ellipsoid:L:a:b:c', 'torus:nu:nv:R:r' or 'dziuk:L'."""
    parts = spec.split(":")
    kind = parts[0]
    if kind == "dziuk":
        return dziuk(int(parts[1]))
    if kind == "sphere":
        return icosphere(int(parts[1]))
    if kind == "ellipsoid":
        return ellipsoid(int(parts[1]), float(parts[2]), float(parts[3]), float(parts[4]))
    if kind == "torus":
        return torus(int(parts[1]), int(parts[2]), float(parts[3]), float(parts[4]))
    raise ValueError(f"unknown mesh spec {spec!r}")
