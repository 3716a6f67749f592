// Triangulated surfaces Gamma_h (Sec. 2.1): validation and the generators of
// the icosphere and the torus.  Vertex and triangle order follow one fixed
// rule (the icosahedron's 12 vertices, then per refinement level the edge
// midpoints in increasing (min endpoint, max endpoint) order), so meshes made
// here and meshes made by other tools with the same rule coincide.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "seg_internal.h"

namespace segimpl {

std::string validate_mesh(const HostMesh& m, seg_status* code) {
  char buf[256];
  if (m.n < 3 || m.f < 1) {
    *code = SEG_ERR_ARG;
    return "mesh needs at least 3 vertices and 1 triangle";
  }
  for (int64_t i = 0; i < 3 * m.n; ++i) {
    if (!std::isfinite(m.xyz[i])) {
      *code = SEG_ERR_ARG;
      snprintf(buf, sizeof buf, "vertex coordinate %lld is not finite", (long long)(i / 3));
      return buf;
    }
  }
  for (int64_t t = 0; t < m.f; ++t) {
    const int32_t* v = &m.tri[3 * t];
    for (int k = 0; k < 3; ++k) {
      if (v[k] < 0 || v[k] >= m.n) {
        *code = SEG_ERR_ARG;
        snprintf(buf, sizeof buf, "triangle %lld has vertex index %d outside [0, %lld)", (long long)t,
                 v[k], (long long)m.n);
        return buf;
      }
    }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) {
      *code = SEG_ERR_MESH;
      snprintf(buf, sizeof buf, "triangle %lld repeats a vertex", (long long)t);
      return buf;
    }
    const double* a = &m.xyz[3 * v[0]];
    const double* b = &m.xyz[3 * v[1]];
    const double* c = &m.xyz[3 * v[2]];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    double twice_area = std::sqrt(cx * cx + cy * cy + cz * cz);
    double scale = (e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) +
                   (e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    if (!(twice_area > 1e-14 * scale)) {
      *code = SEG_ERR_MESH;
      snprintf(buf, sizeof buf, "triangle %lld has zero area", (long long)t);
      return buf;
    }
  }
  *code = SEG_OK;
  return "";
}

static void normalise3(double* p) {
  double s = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  p[0] /= s;
  p[1] /= s;
  p[2] /= s;
}

void make_icosphere(int level, HostMesh* out) {
  const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
  std::vector<double> xyz;
  for (double s1 : {-1.0, 1.0}) {
    for (double s2 : {-1.0, 1.0}) {
      double p[3][3] = {{0.0, s1, s2 * phi}, {s1, s2 * phi, 0.0}, {s2 * phi, 0.0, s1}};
      for (auto& q : p) xyz.insert(xyz.end(), q, q + 3);
    }
  }
  const int n0 = 12;
  auto d2 = [&](int a, int b) {
    double s = 0;
    for (int k = 0; k < 3; ++k) s += (xyz[3 * a + k] - xyz[3 * b + k]) * (xyz[3 * a + k] - xyz[3 * b + k]);
    return s;
  };
  auto adj = [&](int a, int b) { return std::fabs(d2(a, b) - 4.0) < 1e-9; };
  std::vector<int32_t> tri;
  for (int a = 0; a < n0; ++a)
    for (int b = a + 1; b < n0; ++b) {
      if (!adj(a, b)) continue;
      for (int c = b + 1; c < n0; ++c) {
        if (!(adj(a, c) && adj(b, c))) continue;
        const double* A = &xyz[3 * a];
        const double* B = &xyz[3 * b];
        const double* C = &xyz[3 * c];
        double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double nx = e1[1] * e2[2] - e1[2] * e2[1];
        double ny = e1[2] * e2[0] - e1[0] * e2[2];
        double nz = e1[0] * e2[1] - e1[1] * e2[0];
        double dot = nx * (A[0] + B[0] + C[0]) + ny * (A[1] + B[1] + C[1]) + nz * (A[2] + B[2] + C[2]);
        if (dot > 0) {
          tri.insert(tri.end(), {a, b, c});
        } else {
          tri.insert(tri.end(), {a, c, b});
        }
      }
    }
  for (int v = 0; v < n0; ++v) normalise3(&xyz[3 * v]);

  for (int l = 0; l < level; ++l) {
    const int64_t n = (int64_t)xyz.size() / 3;
    const int64_t f = (int64_t)tri.size() / 3;
    std::vector<int64_t> keys(3 * f);
    for (int64_t t = 0; t < f; ++t) {
      for (int k = 0; k < 3; ++k) {
        int64_t a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3];
        int64_t lo = std::min(a, b), hi = std::max(a, b);
        keys[k * f + t] = lo * n + hi;  // edge k of triangle t: (a,b), (b,c), (c,a)
      }
    }
    std::vector<int64_t> ukeys(keys);
    std::sort(ukeys.begin(), ukeys.end());
    ukeys.erase(std::unique(ukeys.begin(), ukeys.end()), ukeys.end());
    const int64_t ne = (int64_t)ukeys.size();
    std::vector<double> nxyz(3 * (n + ne));
    std::copy(xyz.begin(), xyz.end(), nxyz.begin());
    for (int64_t e = 0; e < ne; ++e) {
      int64_t lo = ukeys[e] / n, hi = ukeys[e] % n;
      double* p = &nxyz[3 * (n + e)];
      for (int k = 0; k < 3; ++k) p[k] = xyz[3 * lo + k] + xyz[3 * hi + k];
      normalise3(p);
    }
    auto mid = [&](int64_t key) {
      return (int32_t)(n + (std::lower_bound(ukeys.begin(), ukeys.end(), key) - ukeys.begin()));
    };
    std::vector<int32_t> ntri(12 * f);
    for (int64_t t = 0; t < f; ++t) {
      int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
      int32_t ab = mid(keys[t]), bc = mid(keys[f + t]), ca = mid(keys[2 * f + t]);
      int32_t blocks[4][3] = {{a, ab, ca}, {b, bc, ab}, {c, ca, bc}, {ab, bc, ca}};
      for (int q = 0; q < 4; ++q)
        for (int k = 0; k < 3; ++k) ntri[3 * (q * f + t) + k] = blocks[q][k];
    }
    xyz.swap(nxyz);
    tri.swap(ntri);
  }
  out->xyz.swap(xyz);
  out->tri.swap(tri);
  out->n = (int64_t)out->xyz.size() / 3;
  out->f = (int64_t)out->tri.size() / 3;
}

void make_torus(int nu, int nv, double R, double r, HostMesh* out) {
  out->n = (int64_t)nu * nv;
  out->f = 2 * (int64_t)nu * nv;
  out->xyz.assign(3 * out->n, 0.0);
  out->tri.assign(3 * out->f, 0);
  for (int j = 0; j < nu; ++j) {
    double u = 2.0 * M_PI * j / nu;
    for (int k = 0; k < nv; ++k) {
      double v = 2.0 * M_PI * k / nv;
      double rho = R + r * std::cos(v);
      double* p = &out->xyz[3 * ((int64_t)j * nv + k)];
      p[0] = rho * std::cos(u);
      p[1] = rho * std::sin(u);
      p[2] = r * std::sin(v);
    }
  }
  const int64_t half = (int64_t)nu * nv;
  for (int j = 0; j < nu; ++j) {
    for (int k = 0; k < nv; ++k) {
      int64_t q = (int64_t)j * nv + k;
      int32_t v00 = j * nv + k, v10 = ((j + 1) % nu) * nv + k;
      int32_t v11 = ((j + 1) % nu) * nv + (k + 1) % nv, v01 = j * nv + (k + 1) % nv;
      int32_t* t1 = &out->tri[3 * q];
      int32_t* t2 = &out->tri[3 * (half + q)];
      t1[0] = v00; t1[1] = v10; t1[2] = v11;
      t2[0] = v00; t2[1] = v11; t2[2] = v01;
    }
  }
}

}  // namespace segimpl
