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

static void make_icosahedral(int level, bool dziuk, HostMesh* out) {
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

  HostMesh m;
  m.xyz.swap(xyz);
  m.tri.swap(tri);
  m.n = (int64_t)m.xyz.size() / 3;
  m.f = (int64_t)m.tri.size() / 3;
  if (dziuk) {
    for (int64_t v = 0; v < m.n; ++v) project_point(&m.xyz[3 * v], SurfaceDesc{SEG_SURFACE_DZIUK, 0, 0, 0});
  }
  const SurfaceDesc surf{dziuk ? SEG_SURFACE_DZIUK : SEG_SURFACE_ELLIPSOID, 1.0, 1.0, 1.0};
  for (int l = 0; l < level; ++l) {
    HostMesh fine;
    refine_mesh(m, surf, &fine, nullptr);
    m = std::move(fine);
  }
  *out = std::move(m);
}

void make_icosphere(int level, HostMesh* out) { make_icosahedral(level, false, out); }
void make_dziuk(int level, HostMesh* out) { make_icosahedral(level, true, out); }

void project_point(double* p, const SurfaceDesc& s) {
  switch (s.kind) {
    case SEG_SURFACE_ELLIPSOID: {
      const double q0 = p[0] / s.p0, q1 = p[1] / s.p1, q2 = p[2] / s.p2;
      const double q = std::sqrt(q0 * q0 + q1 * q1 + q2 * q2);
      for (int k = 0; k < 3; ++k) p[k] /= q;
      break;
    }
    case SEG_SURFACE_TORUS: {
      // closest point: the nearest point of the core circle of radius R, then
      // distance r from it towards p
      const double R = s.p0, r = s.p1;
      const double rho = std::sqrt(p[0] * p[0] + p[1] * p[1]);
      const double c[3] = {R * p[0] / rho, R * p[1] / rho, 0.0};
      const double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
      const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int k = 0; k < 3; ++k) p[k] = c[k] + r * d[k] / dn;
      break;
    }
    case SEG_SURFACE_DZIUK: {
      // Newton projection onto Phi = 0 along the gradient:
      // x <- x - Phi(x) grad Phi(x) / |grad Phi(x)|^2 until |Phi| <= 1e-14
      for (int it = 0; it < 50; ++it) {
        const double w = p[0] - p[2] * p[2];
        const double phi = w * w + p[1] * p[1] + p[2] * p[2] - 1.0;
        if (!(std::fabs(phi) > 1e-14)) break;
        const double g[3] = {2.0 * w, 2.0 * p[1], 2.0 * p[2] - 4.0 * p[2] * w};
        const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const double f = phi / g2;
        for (int k = 0; k < 3; ++k) p[k] -= f * g[k];
      }
      break;
    }
    default:
      break;  // SEG_SURFACE_NONE: keep the point
  }
}

void refine_mesh(const HostMesh& in, const SurfaceDesc& surf, HostMesh* out, std::vector<int32_t>* parents) {
  const int64_t n = in.n, f = in.f;
  std::vector<int64_t> keys(3 * f);
  for (int64_t t = 0; t < f; ++t) {
    for (int k = 0; k < 3; ++k) {
      int64_t a = in.tri[3 * t + k], b = in.tri[3 * t + (k + 1) % 3];
      int64_t lo = std::min(a, b), hi = std::max(a, b);
      keys[k * f + t] = lo * n + hi;  // edge k of triangle t: (a,b), (b,c), (c,a)
    }
  }
  std::vector<int64_t> ukeys(keys);
  std::sort(ukeys.begin(), ukeys.end());
  ukeys.erase(std::unique(ukeys.begin(), ukeys.end()), ukeys.end());
  const int64_t ne = (int64_t)ukeys.size();
  HostMesh m;
  m.n = n + ne;
  m.f = 4 * f;
  m.xyz.resize(3 * m.n);
  std::copy(in.xyz.begin(), in.xyz.end(), m.xyz.begin());
  if (parents) {
    parents->resize(2 * m.n);
    for (int64_t v = 0; v < n; ++v) (*parents)[2 * v] = (*parents)[2 * v + 1] = (int32_t)v;
  }
  for (int64_t e = 0; e < ne; ++e) {
    const int64_t lo = ukeys[e] / n, hi = ukeys[e] % n;
    double* p = &m.xyz[3 * (n + e)];
    for (int k = 0; k < 3; ++k) p[k] = 0.5 * (in.xyz[3 * lo + k] + in.xyz[3 * hi + k]);
    project_point(p, surf);
    if (parents) {
      (*parents)[2 * (n + e)] = (int32_t)lo;
      (*parents)[2 * (n + e) + 1] = (int32_t)hi;
    }
  }
  auto mid = [&](int64_t key) {
    return (int32_t)(n + (std::lower_bound(ukeys.begin(), ukeys.end(), key) - ukeys.begin()));
  };
  m.tri.resize(12 * f);
  for (int64_t t = 0; t < f; ++t) {
    int32_t a = in.tri[3 * t], b = in.tri[3 * t + 1], c = in.tri[3 * t + 2];
    int32_t ab = mid(keys[t]), bc = mid(keys[f + t]), ca = mid(keys[2 * f + t]);
    int32_t blocks[4][3] = {{a, ab, ca}, {b, bc, ab}, {c, ca, bc}, {ab, bc, ca}};
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < 3; ++k) m.tri[3 * (q * f + t) + k] = blocks[q][k];
  }
  *out = std::move(m);
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
