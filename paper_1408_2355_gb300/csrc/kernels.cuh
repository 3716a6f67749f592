// Hot-path kernels of one step of Algorithm 2.2 on interleaved vertex rows.
//
// Data layout: every vector is X[row][ms] (vertex-major, ms = m padded to a
// multiple of 16 bytes / sizeof(T)); one row is split across LPR lanes, each
// lane owning VW = 16 / sizeof(T) consecutive components that it moves with
// one 128-bit load or store.  A warp therefore covers 32 / LPR rows, and one
// read of a CSR row (column index + value) serves all m components.
//
// Per step the kernels run in this order (one CUDA graph per step, the CG
// loop is a device-controlled conditional WHILE node):
//   k_start   r0 = -tau K X (warm start x0 = X: M X - A X = -tau K X), and the
//             per-component sums ||X||_M^2, ||M X||^2, X^T K X, r.D^-1 r, r.r
//             -- the normalisation of the previous step (step 3) is fused here
//   k_energy  (every check_every steps) S_eps and the coupling integrals
//   k_cg_a    p = D^-1 r + beta p_old, q = A p, p.q; lagged x += alpha p_old
//   k_cg_b    r -= alpha q, r.D^-1 r, r.r; convergence and beta
//   k_finish  last x += alpha p, then the exact nodal ODE of step 2
//
// Inner products are per component.  For float data each lane accumulates
// the exact products (Dekker split with fma) in a float-float pair, the warp,
// block and grid reductions add float-float pairs, and the final value is a
// float64; for double data everything is float64.  The grid reduction is done
// by the last block to finish (ticket counter), in a fixed order, so results
// are bitwise reproducible for a fixed launch geometry.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "seg_internal.h"

namespace segimpl {

template <typename T>
struct VecW;
template <>
struct VecW<float> {
  static constexpr int W = 4;
};
template <>
struct VecW<double> {
  static constexpr int W = 2;
};

__device__ __forceinline__ void ld(float (&d)[4], const float* p) {
  float4 x = *reinterpret_cast<const float4*>(p);
  d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
}
__device__ __forceinline__ void ld_ro(float (&d)[4], const float* p) {
  float4 x = __ldg(reinterpret_cast<const float4*>(p));
  d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
}
__device__ __forceinline__ void st(float* p, const float (&d)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
}
__device__ __forceinline__ void ld(double (&d)[2], const double* p) {
  double2 x = *reinterpret_cast<const double2*>(p);
  d[0] = x.x; d[1] = x.y;
}
__device__ __forceinline__ void ld_ro(double (&d)[2], const double* p) {
  double2 x = __ldg(reinterpret_cast<const double2*>(p));
  d[0] = x.x; d[1] = x.y;
}
__device__ __forceinline__ void st(double* p, const double (&d)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(d[0], d[1]);
}

__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }

// ------------------------------------------------------------ accumulators

// Float-float accumulator: (hi, lo) with hi + lo the running sum.  Products
// are split exactly (p + e == a*b with fma) and added with Knuth's TwoSum.
// The _rn intrinsics keep the compiler from contracting or reassociating.
struct AccF {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void two_sum_into(float b, float b_err) {
    float s = __fadd_rn(hi, b);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, b_err));
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = __fmaf_rn(a, b, -p);
    two_sum_into(p, pe);
  }
  __device__ __forceinline__ void add_val(float a) { two_sum_into(a, 0.f); }
  __device__ __forceinline__ void add_pair(float ohi, float olo) {
    two_sum_into(ohi, olo);
    float s = __fadd_rn(hi, lo);  // renormalise (Fast2Sum)
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

struct AccD {
  double v;
  __device__ __forceinline__ void zero() { v = 0.0; }
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void add_val(double a) { v += a; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename T>
struct AccOf;
template <>
struct AccOf<float> {
  typedef AccF type;
  typedef float2 part;
};
template <>
struct AccOf<double> {
  typedef AccD type;
  typedef double part;
};

__device__ __forceinline__ float2 to_part(const AccF& a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ double to_part(const AccD& a) { return a.v; }
__device__ __forceinline__ void add_part(AccF& a, float2 p) { a.add_pair(p.x, p.y); }
__device__ __forceinline__ void add_part(AccD& a, double p) { a.v += p; }
__device__ __forceinline__ void shfl_add(AccF& a, int off) {
  float h = __shfl_xor_sync(0xffffffffu, a.hi, off);
  float l = __shfl_xor_sync(0xffffffffu, a.lo, off);
  a.add_pair(h, l);
}
__device__ __forceinline__ void shfl_add(AccD& a, int off) { a.v += __shfl_xor_sync(0xffffffffu, a.v, off); }

// Block + grid reduction of ND per-component sums.  Every block writes its
// partial; the last block to arrive sums the partials of all blocks in block
// order and leaves the totals in tot[ND][kMaxCols].  Returns true in the last
// block only.  Must be reached by every block of the grid.
template <typename T, int LPR, int ND>
__device__ __forceinline__ bool grid_reduce(typename AccOf<T>::type (&acc)[ND][VecW<T>::W],
                                            const KArgs<T>& a, int slot, double (*tot)[kMaxCols]) {
  typedef typename AccOf<T>::type Acc;
  typedef typename AccOf<T>::part Part;
  constexpr int VW = VecW<T>::W;
  constexpr int NW = kBlockThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cg = lane % LPR;
#pragma unroll
  for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < VW; ++v) shfl_add(acc[d][v], off);
  __shared__ Part red[ND][NW][kMaxCols];
  __shared__ unsigned int ticket;
  if (lane < LPR) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < VW; ++v) red[d][warp][cg * VW + v] = to_part(acc[d][v]);
  }
  __syncthreads();
  const int G = gridDim.x;
  Part* part = reinterpret_cast<Part*>(a.part);
  for (int t = threadIdx.x; t < ND * a.ms; t += kBlockThreads) {
    const int d = t / a.ms, c = t % a.ms;
    Acc s;
    s.zero();
    for (int w = 0; w < NW; ++w) add_part(s, red[d][w][c]);
    part[(size_t)(d * a.ms + c) * G + blockIdx.x] = to_part(s);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&a.ctl->counters[slot], 1u);
  __syncthreads();
  if (ticket != (unsigned int)(G - 1)) return false;
  __threadfence();
  for (int pidx = warp; pidx < ND * a.ms; pidx += NW) {
    Acc s;
    s.zero();
    for (int b = lane; b < G; b += 32) add_part(s, __ldcg(&part[(size_t)pidx * G + b]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) shfl_add(s, off);
    if (lane == 0) tot[pidx / a.ms][pidx % a.ms] = s.value();
  }
  __syncthreads();
  if (threadIdx.x == 0) a.ctl->counters[slot] = 0u;
  return true;
}

// Exclusive sums over the components of one vertex row held by the LPR lanes
// starting at lane `lbase`: ex[v] = sum of x over all components except v,
// formed as (prefix) + (suffix) of non-negative terms -- no subtraction.
template <typename T, int LPR, int NQ>
__device__ __forceinline__ void row_exclusive(const T (&x)[NQ][VecW<T>::W], T (&ex)[NQ][VecW<T>::W],
                                              int lbase, int cg) {
  constexpr int VW = VecW<T>::W;
  T lt[NQ], pre[NQ], suf[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T s = T(0);
#pragma unroll
    for (int v = 0; v < VW; ++v) s += x[q][v];
    lt[q] = s;
    pre[q] = T(0);
    suf[q] = T(0);
  }
#pragma unroll
  for (int k = 0; k < LPR; ++k) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T o = __shfl_sync(0xffffffffu, lt[q], lbase + k);
      if (k < cg) pre[q] += o;
      if (k > cg) suf[q] += o;
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T in_suf[VW];
    T s = T(0);
#pragma unroll
    for (int v = VW - 1; v >= 0; --v) {
      in_suf[v] = s;
      s += x[q][v];
    }
    T p = pre[q];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      ex[q][v] = p + (in_suf[v] + suf[q]);
      p += x[q][v];
    }
  }
}

// ---------------------------------------------------------------- kernels

#define SEG_ROW_SETUP                                                         \
  constexpr int VW = VecW<T>::W;                                              \
  constexpr int NW = kBlockThreads / 32;                                      \
  constexpr int RPW = 32 / LPR;                                               \
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;                 \
  const int rs = lane / LPR, cg = lane % LPR, c0 = cg * VW;                   \
  (void)rs;                                                                   \
  const int r0 = blockIdx.x * a.rows_per_block;                               \
  const int r1 = min(a.n, r0 + a.rows_per_block);

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlockThreads, 2) k_start(const KArgs<T> a) {
  typedef typename AccOf<T>::type Acc;
  DevCtl* ctl = a.ctl;
  if (ctl->halted && !a.ignore_halt) return;
  SEG_ROW_SETUP
  const T tau = (T)a.tau;
  Acc acc[5][VW];
#pragma unroll
  for (int d = 0; d < 5; ++d)
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[d][v].zero();
  for (int base = r0 + warp * RPW; base < r1; base += NW * RPW) {
    const int row = base + rs;
    if (row < r1) {
      T x[VW], kx[VW], mx[VW];
      ld(x, a.X + (size_t)row * a.ms + c0);
#pragma unroll
      for (int v = 0; v < VW; ++v) kx[v] = mx[v] = T(0);
      const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const int j = __ldg(a.col + e);
        const T kv = __ldg(a.valK + e), mv = __ldg(a.valM + e);
        T xj[VW];
        ld(xj, a.X + (size_t)j * a.ms + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          kx[v] = fma(kv, xj[v], kx[v]);
          mx[v] = fma(mv, xj[v], mx[v]);
        }
      }
      const T di = __ldg(a.dinv + row);
      T r[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) r[v] = -tau * kx[v];
      st(a.R + (size_t)row * a.ms + c0, r);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        acc[0][v].add_prod(x[v], mx[v]);
        acc[1][v].add_prod(mx[v], mx[v]);
        acc[2][v].add_prod(x[v], kx[v]);
        acc[3][v].add_prod(r[v], di * r[v]);
        acc[4][v].add_prod(r[v], r[v]);
      }
    }
  }
  __shared__ double tot[5][kMaxCols];
  if (!grid_reduce<T, LPR, 5>(acc, a, kCtrStart, tot)) return;
  int act = 0, bad = 0;
  const int c = threadIdx.x;
  if (c < a.ms) {
    const double n2 = tot[0][c], bb = tot[1][c], ukt = tot[2][c], rz = tot[3][c], rr = tot[4][c];
    const bool real = c < a.m;
    if (real && !(n2 > 0.0 && isfinite(n2) && isfinite(rr) && isfinite(ukt))) bad = 1;
    ctl->n2[c] = n2;
    ctl->inv_n[c] = (real && n2 > 0.0) ? 1.0 / sqrt(n2) : 0.0;
    ctl->lam[c] = (real && n2 > 0.0) ? ukt / n2 : 0.0;
    ctl->tol2[c] = a.rtol2 * bb;
    ctl->rz[c] = rz;
    ctl->alpha[0][c] = 0.0;
    ctl->alpha[1][c] = 0.0;
    ctl->beta[c] = 0.0;
    act = (real && !bad && rr > a.rtol2 * bb) ? 1 : 0;
    ctl->active[c] = act;
  }
  const int any = __syncthreads_or(act);
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    ctl->it = 0;
    int cont = (any && !anybad) ? 1 : 0;
    if (anybad) {
      ctl->status |= 2;
      ctl->halted = 2;
    }
    ctl->cont = cont;
    if (a.set_cond) cudaGraphSetConditional(a.cond, cont);
  }
}

// S_eps and the per-component coupling integrals c_i = int u_i^2 e_i with
// e_i = sum_{j != i} u_j^2, integrated exactly on every flat triangle.  With
// a = (u_i at the 3 corners) and B = sum_{j != i} a_j a_j^T, the moments of
// the barycentric coordinates give
//   int_T (a.lam)^2 (lam^T B lam) = |T|/360 [ (s^2 + |a|^2)(1^T B 1 + tr B)
//        + 4 s a^T B 1 + 2 a^T B a + 4 (a o a)^T B 1 + 4 s a^T diag(B)
//        + 6 (a o a)^T diag(B) ],   s = a_0 + a_1 + a_2.
template <typename T, int LPR>
__global__ void __launch_bounds__(kBlockThreads, 2) k_energy(const KArgs<T> a) {
  typedef typename AccOf<T>::type Acc;
  constexpr int VW = VecW<T>::W;
  constexpr int NW = kBlockThreads / 32;
  constexpr int RPW = 32 / LPR;
  DevCtl* ctl = a.ctl;
  if (ctl->halted && !a.ignore_halt) return;
  if (!a.force) {
    if (a.check_every <= 0) return;
    if (ctl->step % a.check_every != 0) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rs = lane / LPR, cg = lane % LPR, c0 = cg * VW, lbase = lane - cg;
  const int t0 = blockIdx.x * a.tri_per_block;
  const int t1 = min(a.ntri, t0 + a.tri_per_block);
  T invn[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) invn[v] = (T)ctl->inv_n[c0 + v];
  Acc acc[1][VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[0][v].zero();
  const T inv360 = T(1) / T(360);
  for (int base = t0 + warp * RPW; base < t1; base += NW * RPW) {
    const int t = base + rs;
    const bool valid = t < t1;
    T u[3][VW];
    T area = T(0);
    if (valid) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int row = __ldg(a.tri + 3 * t + k);
        ld(u[k], a.X + (size_t)row * a.ms + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) u[k][v] *= invn[v];
      }
      area = __ldg(a.tarea + t);
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int v = 0; v < VW; ++v) u[k][v] = T(0);
    }
    // P = a a^T per component: 00, 11, 22, 01, 02, 12
    T P[6][VW], E[6][VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      P[0][v] = u[0][v] * u[0][v];
      P[1][v] = u[1][v] * u[1][v];
      P[2][v] = u[2][v] * u[2][v];
      P[3][v] = u[0][v] * u[1][v];
      P[4][v] = u[0][v] * u[2][v];
      P[5][v] = u[1][v] * u[2][v];
    }
    row_exclusive<T, LPR, 6>(P, E, lbase, cg);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const T a0 = u[0][v], a1 = u[1][v], a2 = u[2][v];
      const T e00 = E[0][v], e11 = E[1][v], e22 = E[2][v], e01 = E[3][v], e02 = E[4][v], e12 = E[5][v];
      const T s = a0 + a1 + a2;
      const T q0 = a0 * a0, q1 = a1 * a1, q2 = a2 * a2;
      const T aa = q0 + q1 + q2;
      const T b1x = e00 + e01 + e02, b1y = e01 + e11 + e12, b1z = e02 + e12 + e22;
      const T SB = b1x + b1y + b1z, trB = e00 + e11 + e22;
      const T aB1 = a0 * b1x + a1 * b1y + a2 * b1z;
      const T aBa = q0 * e00 + q1 * e11 + q2 * e22 + T(2) * (a0 * a1 * e01 + a0 * a2 * e02 + a1 * a2 * e12);
      const T a2B1 = q0 * b1x + q1 * b1y + q2 * b1z;
      const T dBa = a0 * e00 + a1 * e11 + a2 * e22;
      const T a2dB = q0 * e00 + q1 * e11 + q2 * e22;
      const T F = (s * s + aa) * (SB + trB) + T(4) * s * aB1 + T(2) * aBa + T(4) * a2B1 + T(4) * s * dBa +
                  T(6) * a2dB;
      acc[0][v].add_val(area * inv360 * F);
    }
  }
  __shared__ double tot[1][kMaxCols];
  if (!grid_reduce<T, LPR, 1>(acc, a, kCtrEnergy, tot)) return;
  if (threadIdx.x < a.ms) ctl->coup[threadIdx.x] = threadIdx.x < a.m ? tot[0][threadIdx.x] : 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, D = 0.0;
    for (int c = 0; c < a.m; ++c) {
      S += tot[0][c];
      D += ctl->lam[c];
    }
    S *= a.inv_eps2;
    const double total = D + S;
    ctl->e_total = total;
    ctl->e_dir = D;
    ctl->e_s = S;
    if (!a.force) {
      ctl->checks += 1;
      int stop = 0;
      if (!isfinite(total)) {
        ctl->status |= 2;
        ctl->halted = 2;
        stop = 1;
      } else {
        if (ctl->have_prev && a.energy_tol >= 0.0 && fabs(total - ctl->e_prev) < a.energy_tol) {
          ctl->halted = 1;
          stop = 1;
        }
        ctl->e_prev = total;
        ctl->have_prev = 1;
      }
      if (stop) {
        ctl->cont = 0;
        if (a.set_cond) cudaGraphSetConditional(a.cond, 0);
      }
    }
  }
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlockThreads, 2) k_cg_a(const KArgs<T> a) {
  typedef typename AccOf<T>::type Acc;
  DevCtl* ctl = a.ctl;
  if (ctl->halted && !a.ignore_halt) return;
  SEG_ROW_SETUP
  const int it = ctl->it;
  const T* Pold = (it & 1) ? a.P1 : a.P0;
  T* Pnew = (it & 1) ? a.P0 : a.P1;
  T beta[VW], alx[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    beta[v] = (T)ctl->beta[c0 + v];
    alx[v] = (T)ctl->alpha[it & 1][c0 + v];
  }
  Acc acc[1][VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[0][v].zero();
  for (int base = r0 + warp * RPW; base < r1; base += NW * RPW) {
    const int row = base + rs;
    if (row < r1) {
      const size_t off = (size_t)row * a.ms + c0;
      T ri[VW], po[VW], x[VW], pn[VW], q[VW];
      ld_ro(ri, a.R + off);
      ld_ro(po, Pold + off);
      ld(x, a.X + off);
      const T di = __ldg(a.dinv + row);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        pn[v] = fma(beta[v], po[v], di * ri[v]);
        x[v] = fma(alx[v], po[v], x[v]);
        q[v] = T(0);
      }
      st(a.X + off, x);
      const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const int j = __ldg(a.col + e);
        const T av = __ldg(a.valA + e);
        const T dj = __ldg(a.dinv + j);
        const size_t oj = (size_t)j * a.ms + c0;
        T rj[VW], pj[VW];
        ld_ro(rj, a.R + oj);
        ld_ro(pj, Pold + oj);
#pragma unroll
        for (int v = 0; v < VW; ++v) q[v] = fma(av, fma(beta[v], pj[v], dj * rj[v]), q[v]);
      }
      st(Pnew + off, pn);
      st(a.Q + off, q);
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[0][v].add_prod(pn[v], q[v]);
    }
  }
  __shared__ double tot[1][kMaxCols];
  if (!grid_reduce<T, LPR, 1>(acc, a, kCtrCgA, tot)) return;
  const int c = threadIdx.x;
  if (c < a.ms) {
    const double pq = tot[0][c];
    ctl->alpha[(it + 1) & 1][c] = (ctl->active[c] && pq > 0.0) ? ctl->rz[c] / pq : 0.0;
  }
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlockThreads, 2) k_cg_b(const KArgs<T> a) {
  typedef typename AccOf<T>::type Acc;
  DevCtl* ctl = a.ctl;
  if (ctl->halted && !a.ignore_halt) return;
  SEG_ROW_SETUP
  const int it = ctl->it;
  T al[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) al[v] = (T)ctl->alpha[(it + 1) & 1][c0 + v];
  Acc acc[2][VW];
#pragma unroll
  for (int d = 0; d < 2; ++d)
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[d][v].zero();
  for (int base = r0 + warp * RPW; base < r1; base += NW * RPW) {
    const int row = base + rs;
    if (row < r1) {
      const size_t off = (size_t)row * a.ms + c0;
      T r[VW], q[VW];
      ld(r, a.R + off);
      ld_ro(q, a.Q + off);
      const T di = __ldg(a.dinv + row);
#pragma unroll
      for (int v = 0; v < VW; ++v) r[v] = fma(-al[v], q[v], r[v]);
      st(a.R + off, r);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        acc[0][v].add_prod(r[v], di * r[v]);
        acc[1][v].add_prod(r[v], r[v]);
      }
    }
  }
  __shared__ double tot[2][kMaxCols];
  if (!grid_reduce<T, LPR, 2>(acc, a, kCtrCgB, tot)) return;
  int act = 0, bad = 0;
  const int c = threadIdx.x;
  if (c < a.ms) {
    const double rzn = tot[0][c], rrn = tot[1][c];
    act = ctl->active[c];
    if (c < a.m && !(isfinite(rzn) && isfinite(rrn))) bad = 1;
    if (act && rrn <= ctl->tol2[c]) act = 0;
    const double rzo = ctl->rz[c];
    ctl->beta[c] = rzo > 0.0 ? rzn / rzo : 0.0;
    ctl->rz[c] = rzn;
    ctl->active[c] = act;
  }
  const int any = __syncthreads_or(act);
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    const int it1 = it + 1;
    ctl->it = it1;
    int cont = (any && it1 < a.maxit) ? 1 : 0;
    if (any && it1 >= a.maxit) ctl->status |= 1;
    if (anybad) {
      ctl->status |= 2;
      ctl->halted = 2;
      cont = 0;
    }
    ctl->cont = cont;
    if (a.set_cond) cudaGraphSetConditional(a.cond, cont);
  }
}

// Last CG update x += alpha p (lagged from the final iteration), then the
// exact solution of the nodal ODE of step 2 (Jacobi form):
//   u~ = x * inv_n,  u^_i = u~_i exp(-(2 tau/eps^2) sum_{j != i} u~_j^2).
template <typename T, int LPR>
__global__ void __launch_bounds__(kBlockThreads, 2) k_finish(const KArgs<T> a) {
  DevCtl* ctl = a.ctl;
  if (ctl->halted && !a.ignore_halt) return;
  SEG_ROW_SETUP
  const int lbase = lane - cg;
  const int it = ctl->it;
  const T* P = (it & 1) ? a.P1 : a.P0;
  T al[VW], invn[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    al[v] = a.apply_x ? (T)ctl->alpha[it & 1][c0 + v] : T(0);
    invn[v] = (T)ctl->inv_n[c0 + v];
  }
  const T mcoef = -(T)a.coef;
  for (int base = r0 + warp * RPW; base < r1; base += NW * RPW) {
    const int row = base + rs;
    const bool valid = row < r1;
    const size_t off = (size_t)row * a.ms + c0;
    T x[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) x[v] = T(0);
    if (valid) {
      ld(x, a.X + off);
      if (a.apply_x) {
        T p[VW];
        ld_ro(p, P + off);
#pragma unroll
        for (int v = 0; v < VW; ++v) x[v] = fma(al[v], p[v], x[v]);
      }
    }
    if (a.apply_ode) {
      T sq[1][VW], ex[1][VW], ut[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        ut[v] = x[v] * invn[v];
        sq[0][v] = ut[v] * ut[v];
      }
      row_exclusive<T, LPR, 1>(sq, ex, lbase, cg);
#pragma unroll
      for (int v = 0; v < VW; ++v) x[v] = ut[v] * t_exp(mcoef * ex[0][v]);
    }
    if (valid) st(a.X + off, x);
  }
  if (a.count_step && blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->step += 1;
    ctl->cg_last = it;
    ctl->cg_total += it;
    if (it > ctl->cg_max) ctl->cg_max = it;
  }
}

// ------------------------------------------------------- auxiliary kernels

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long seed, long long z, int m, int i) {
  unsigned long long ctr = (unsigned long long)z * (unsigned long long)m + (unsigned long long)i;
  unsigned long long h = splitmix64(seed ^ splitmix64(ctr));
  return (double)(h >> 11) * 0x1.0p-53;
}

// Sec. 2.2 random initial values (un-normalised) for caller vertex perm[row].
template <typename T>
__global__ void k_init_rng(const KArgs<T> a, const int* perm, unsigned long long seed, int kind) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)a.n * a.ms) return;
  const int row = (int)(idx / a.ms), c = (int)(idx % a.ms);
  const long long z = perm[row];
  double val = 0.0;
  if (c < a.m) {
    if (kind == SEG_INIT_UNIFORM) {
      val = uniform01(seed, z, a.m, c);
    } else {
      int ch = (int)floor((double)a.m * uniform01(seed, z, a.m, 0));
      if (ch > a.m - 1) ch = a.m - 1;
      val = (c == ch) ? 1.0 : 0.0;
    }
  }
  a.X[idx] = (T)val;
}

template <typename T>
__global__ void k_scatter_in(const KArgs<T> a, const double* src, const int* perm) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)a.n * a.ms) return;
  const int row = (int)(idx / a.ms), c = (int)(idx % a.ms);
  a.X[idx] = c < a.m ? (T)src[(long long)perm[row] * a.m + c] : T(0);
}

template <typename T>
__global__ void k_gather_out(const KArgs<T> a, double* dst, const int* iperm) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)a.n * a.m) return;
  const long long z = idx / a.m;
  const int c = (int)(idx % a.m);
  const int row = iperm[z];
  dst[idx] = (double)a.X[(size_t)row * a.ms + c] * a.ctl->inv_n[c];
}

// Partition read-out (eq. (vi)): argmax with the lowest index on ties, and
// v_i = u_i - sum_{j != i} u_j > 0 for that i.
template <typename T>
__global__ void k_labels(const KArgs<T> a, int* am, unsigned char* vp, const int* iperm) {
  const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= a.n) return;
  const int row = iperm[z];
  const T* x = a.X + (size_t)row * a.ms;
  int best = 0;
  T bv = x[0] * (T)a.ctl->inv_n[0];
  for (int c = 1; c < a.m; ++c) {
    const T u = x[c] * (T)a.ctl->inv_n[c];
    if (u > bv) {
      bv = u;
      best = c;
    }
  }
  T others = T(0);
  for (int c = 0; c < a.m; ++c)
    if (c != best) others += x[c] * (T)a.ctl->inv_n[c];
  am[z] = best;
  vp[z] = (bv - others > T(0)) ? 1 : 0;
}

template <typename T, int LPR>
bool fill_kernels(KernelSet* ks) {
  ks->start = (void*)k_start<T, LPR>;
  ks->cg_a = (void*)k_cg_a<T, LPR>;
  ks->cg_b = (void*)k_cg_b<T, LPR>;
  ks->finish = (void*)k_finish<T, LPR>;
  ks->energy = (void*)k_energy<T, LPR>;
  ks->init_rng = (void*)k_init_rng<T>;
  ks->scatter_in = (void*)k_scatter_in<T>;
  ks->gather_out = (void*)k_gather_out<T>;
  ks->labels = (void*)k_labels<T>;
  return true;
}

}  // namespace segimpl
