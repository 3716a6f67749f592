// P1 mass and stiffness matrices on the triangulated surface (Sec. 2.1),
// assembled in float64 on the host.
//
// On a flat triangle T the P1 element matrices are
//   mass:      |T|/12 on the off-diagonal, |T|/6 on the diagonal;
//   stiffness: the cotangent form -- the entry of the edge (i, j) receives
//              -cot(theta_k)/2 where theta_k is the angle at the corner k
//              opposite that edge, and each diagonal entry is minus the sum of
//              the off-diagonal entries of its row.
//
// Before assembly the vertices are renumbered along a 3-D Morton (Z-order)
// curve of their coordinates so that mesh neighbours have nearby row indices:
// the sparse gathers of the device kernels then hit the same cache lines.
// `perm` maps internal rows to caller vertices, `iperm` the reverse.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "seg_internal.h"

namespace segimpl {

static uint64_t spread21(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

static void morton_order(const HostMesh& mesh, std::vector<int32_t>* perm) {
  const int64_t n = mesh.n;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < n; ++v)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], mesh.xyz[3 * v + k]);
      hi[k] = std::max(hi[k], mesh.xyz[3 * v + k]);
    }
  std::vector<uint64_t> key(n);
  for (int64_t v = 0; v < n; ++v) {
    uint64_t c[3];
    for (int k = 0; k < 3; ++k) {
      double span = hi[k] - lo[k];
      double t = span > 0 ? (mesh.xyz[3 * v + k] - lo[k]) / span : 0.0;
      c[k] = (uint64_t)std::min(2097151.0, std::max(0.0, t * 2097151.0));
    }
    key[v] = spread21(c[0]) | spread21(c[1]) << 1 | spread21(c[2]) << 2;
  }
  perm->resize(n);
  std::iota(perm->begin(), perm->end(), 0);
  std::stable_sort(perm->begin(), perm->end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
}

void assemble_p1(const HostMesh& mesh, HostCSR* out) {
  const int64_t n = mesh.n, f = mesh.f;
  morton_order(mesh, &out->perm);
  out->iperm.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) out->iperm[out->perm[i]] = (int32_t)i;

  // triangles in internal numbering, ordered by their smallest row
  std::vector<int32_t> tr(3 * f);
  for (int64_t t = 0; t < 3 * f; ++t) tr[t] = out->iperm[mesh.tri[t]];
  std::vector<int64_t> torder(f);
  std::iota(torder.begin(), torder.end(), 0);
  auto tmin = [&](int64_t t) { return std::min(tr[3 * t], std::min(tr[3 * t + 1], tr[3 * t + 2])); };
  std::stable_sort(torder.begin(), torder.end(), [&](int64_t a, int64_t b) { return tmin(a) < tmin(b); });
  out->tri_rows.resize(3 * f);
  out->area.resize(f);

  // sparsity pattern: the vertex itself and its edge neighbours, sorted
  std::vector<int64_t> deg(n + 1, 0);
  for (int64_t t = 0; t < f; ++t)
    for (int k = 0; k < 3; ++k) deg[tr[3 * t + k]] += 2;
  std::vector<int64_t> start(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + deg[i] + 1;
  std::vector<int32_t> cand(start[n]);
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t i = 0; i < n; ++i) cand[fill[i]++] = (int32_t)i;
  for (int64_t t = 0; t < f; ++t)
    for (int k = 0; k < 3; ++k) {
      int32_t a = tr[3 * t + k], b = tr[3 * t + (k + 1) % 3];
      cand[fill[a]++] = b;
      cand[fill[b]++] = a;
    }
  out->rowptr.assign(n + 1, 0);
  out->col.clear();
  out->col.reserve(7 * n + 16);
  for (int64_t i = 0; i < n; ++i) {
    auto b = cand.begin() + start[i], e = cand.begin() + fill[i];
    std::sort(b, e);
    auto u = std::unique(b, e);
    out->col.insert(out->col.end(), b, u);
    out->rowptr[i + 1] = (int32_t)out->col.size();
  }
  out->n = n;
  out->nnz = (int64_t)out->col.size();
  out->M.assign(out->nnz, 0.0);
  out->K.assign(out->nnz, 0.0);

  auto slot = [&](int32_t i, int32_t j) {
    auto b = out->col.begin() + out->rowptr[i], e = out->col.begin() + out->rowptr[i + 1];
    return (int64_t)(std::lower_bound(b, e, j) - out->col.begin());
  };

  for (int64_t q = 0; q < f; ++q) {
    const int64_t t = torder[q];
    const int32_t v[3] = {tr[3 * t], tr[3 * t + 1], tr[3 * t + 2]};
    for (int k = 0; k < 3; ++k) out->tri_rows[3 * q + k] = v[k];
    const double* x[3];
    for (int k = 0; k < 3; ++k) x[k] = &mesh.xyz[3 * (int64_t)out->perm[v[k]]];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = x[1][d] - x[0][d];
      e2[d] = x[2][d] - x[0][d];
    }
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    const double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    out->area[q] = area;
    for (int k = 0; k < 3; ++k) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;  // edge (i, j) opposite corner k
      double a[3], b[3];
      for (int d = 0; d < 3; ++d) {
        a[d] = x[i][d] - x[k][d];
        b[d] = x[j][d] - x[k][d];
      }
      double dot = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
      double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
      double half_cot = 0.5 * dot / std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
      out->K[slot(v[i], v[j])] -= half_cot;
      out->K[slot(v[j], v[i])] -= half_cot;
      out->K[slot(v[i], v[i])] += half_cot;
      out->K[slot(v[j], v[j])] += half_cot;
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) out->M[slot(v[a], v[b])] += (a == b ? area / 6.0 : area / 12.0);
  }
}

}  // namespace segimpl
