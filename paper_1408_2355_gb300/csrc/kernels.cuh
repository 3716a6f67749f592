// Hot-path kernels of one step of Algorithm 2.2 on interleaved vertex rows.
//
// Data layout: every vector is V[row][ms] (vertex-major, ms = m padded to a
// multiple of 16 bytes / sizeof(T)); one row is split across LPR lanes, each
// lane owning VW = 16 / sizeof(T) consecutive components that it moves with
// one 128-bit load or store.  A warp therefore covers 32 / LPR rows, and one
// read of a padded-ELL matrix row (W column indices + W values) serves all m
// components.
//
// Per step the kernels run in this order (one CUDA graph per step: the first
// CG iterations as plain nodes, the rest in a device-controlled conditional
// WHILE node):
//   k_start         r0 = M X - A (X + y) = -tau K X - A y for the iterate
//                   x = X + y (y: the correction the previous solve ended
//                   with), z0 = D^-1 r0, and the per-component sums
//                   ||X||_M^2, X^T K X, r0.z0, ||M X||^2, ||r0||^2 -- the
//                   renormalisation of the previous step (step 3) is fused here
//   k_energy_check  (every check_every steps) S_eps and the stop rule
//   k_cg_a          p = z + beta p_old, q = A z + beta q_old, p.q; every second
//                   iteration y += the two pending alpha p terms.  In the
//                   first iteration of a solve (p = z) also r.q and q.q, from
//                   which it finds ||r - alpha q|| and ends the solve when
//                   every component has converged
//   k_cg_b          z -= alpha D^-1 q, r.z and r.r (r = D z); convergence, beta
//                   (not needed after a solve that ended in k_cg_a)
//   k_finish        x = X + y with the updates still pending, then the exact
//                   nodal ODE of step 2
// The two gather kernels stage each warp's next groups of rows (ELL indices,
// values and own vector rows) in shared memory with TMA bulk copies while the
// current group's neighbour rows are gathered.
//
// Inner products are per component.  For float data the ones that feed CG's
// alpha / beta, the norms and the energies accumulate the exact products
// (Dekker split with fma) in float-float pairs per lane, the warp, block and
// grid reductions add float-float pairs, and the final value is a float64;
// sums that only set the CG tolerance accumulate in float per lane.  For
// double data everything is float64.  The grid reduction is done by the last
// block to finish (ticket counter), in a fixed order, so results are bitwise
// reproducible for a fixed launch geometry, alone or in a batch.
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
// Loads of state vectors in the step passes: through the read-only cache
// (CO = false) when the launch does not write them, else coherent loads (a
// persistent launch writes them in its earlier phases).
template <bool CO>
__device__ __forceinline__ void ldv(float (&d)[4], const float* p) {
  if constexpr (CO)
    ld(d, p);
  else
    ld_ro(d, p);
}
template <bool CO>
__device__ __forceinline__ void ldv(double (&d)[2], const double* p) {
  if constexpr (CO)
    ld(d, p);
  else
    ld_ro(d, p);
}
// 32-byte loads (one 256-bit load instruction, sm_100 and later; p must be
// 32-byte aligned): read-only (ld_ro32) and coherent (ld32)
// (the "memory" clobber keeps the coherent loads after the grid barrier
// that orders them with the writes of an earlier phase)
__device__ __forceinline__ void ld32(float (&d)[8], const float* p) {
  asm("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]), "=f"(d[6]), "=f"(d[7])
      : "l"(p)
      : "memory");
}
__device__ __forceinline__ void ld32(double (&d)[4], const double* p) {
  asm("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(d[0]), "=d"(d[1]), "=d"(d[2]), "=d"(d[3]) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_ro32(float (&d)[8], const float* p) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]), "=f"(d[6]), "=f"(d[7])
      : "l"(p));
}
__device__ __forceinline__ void ld_ro32(double (&d)[4], const double* p) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(d[0]), "=d"(d[1]), "=d"(d[2]), "=d"(d[3]) : "l"(p));
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

// ------------------------------------------------- packed float32 pairs
// The float passes do the arithmetic of a lane's VW = 4 values as two packed
// pairs (FFMA2 / FADD2 / FMUL2: one instruction per pair, each element
// rounded exactly as the scalar operation would be, so results are bitwise
// those of the scalar code).  For double data the same helpers are scalar.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
// x - y as one rounding of the exact difference (= __fsub_rn)
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, f2(-1.f, -1.f), x); }

// acc[v] += s * x[v]
__device__ __forceinline__ void v_axpy(float (&acc)[4], float s, const float (&x)[4]) {
  const float2 a0 = __ffma2_rn(f2(s, s), f2(x[0], x[1]), f2(acc[0], acc[1]));
  const float2 a1 = __ffma2_rn(f2(s, s), f2(x[2], x[3]), f2(acc[2], acc[3]));
  acc[0] = a0.x; acc[1] = a0.y; acc[2] = a1.x; acc[3] = a1.y;
}
__device__ __forceinline__ void v_axpy(double (&acc)[2], double s, const double (&x)[2]) {
  acc[0] = fma(s, x[0], acc[0]);
  acc[1] = fma(s, x[1], acc[1]);
}
// out[v] = fma(x[v], y[v], z[v])
__device__ __forceinline__ void v_fma(float (&out)[4], const float (&x)[4], const float (&y)[4], const float (&z)[4]) {
  const float2 a0 = __ffma2_rn(f2(x[0], x[1]), f2(y[0], y[1]), f2(z[0], z[1]));
  const float2 a1 = __ffma2_rn(f2(x[2], x[3]), f2(y[2], y[3]), f2(z[2], z[3]));
  out[0] = a0.x; out[1] = a0.y; out[2] = a1.x; out[3] = a1.y;
}
__device__ __forceinline__ void v_fma(double (&out)[2], const double (&x)[2], const double (&y)[2],
                                      const double (&z)[2]) {
  out[0] = fma(x[0], y[0], z[0]);
  out[1] = fma(x[1], y[1], z[1]);
}
// out[v] = s * x[v]
__device__ __forceinline__ void v_scale(float (&out)[4], float s, const float (&x)[4]) {
  const float2 a0 = __fmul2_rn(f2(s, s), f2(x[0], x[1]));
  const float2 a1 = __fmul2_rn(f2(s, s), f2(x[2], x[3]));
  out[0] = a0.x; out[1] = a0.y; out[2] = a1.x; out[3] = a1.y;
}
__device__ __forceinline__ void v_scale(double (&out)[2], double s, const double (&x)[2]) {
  out[0] = s * x[0];
  out[1] = s * x[1];
}
// out[v] = x[v] - y[v]
__device__ __forceinline__ void v_sub(float (&out)[4], const float (&x)[4], const float (&y)[4]) {
  const float2 a0 = sub2(f2(x[0], x[1]), f2(y[0], y[1]));
  const float2 a1 = sub2(f2(x[2], x[3]), f2(y[2], y[3]));
  out[0] = a0.x; out[1] = a0.y; out[2] = a1.x; out[3] = a1.y;
}
__device__ __forceinline__ void v_sub(double (&out)[2], const double (&x)[2], const double (&y)[2]) {
  out[0] = x[0] - y[0];
  out[1] = x[1] - y[1];
}
// Float-float accumulation of two values at once (AccF::add_prod on a pair).
__device__ __forceinline__ void add_prod_pair(AccF& A, AccF& B, float a0, float b0, float a1, float b1) {
  const float2 a = f2(a0, a1), b = f2(b0, b1);
  const float2 p = __fmul2_rn(a, b);
  const float2 pe = __ffma2_rn(a, b, f2(-p.x, -p.y));
  const float2 hi = f2(A.hi, B.hi);
  const float2 s = __fadd2_rn(hi, p);
  const float2 bb = sub2(s, hi);
  const float2 e = __fadd2_rn(sub2(hi, sub2(s, bb)), sub2(p, bb));
  const float2 lo = __fadd2_rn(f2(A.lo, B.lo), __fadd2_rn(e, pe));
  A.hi = s.x; B.hi = s.y; A.lo = lo.x; B.lo = lo.y;
}
// acc[v].add_prod(x[v], y[v])
__device__ __forceinline__ void v_add_prods(AccF (&acc)[4], const float (&x)[4], const float (&y)[4]) {
  add_prod_pair(acc[0], acc[1], x[0], y[0], x[1], y[1]);
  add_prod_pair(acc[2], acc[3], x[2], y[2], x[3], y[3]);
}
__device__ __forceinline__ void v_add_prods(AccD (&acc)[2], const double (&x)[2], const double (&y)[2]) {
  acc[0].add_prod(x[0], y[0]);
  acc[1].add_prod(x[1], y[1]);
}

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
__device__ __forceinline__ float2 plain_part(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ double plain_part(double v) { return v; }
__device__ __forceinline__ void add_part(AccF& a, float2 p) { a.add_pair(p.x, p.y); }
__device__ __forceinline__ void add_part(AccD& a, double p) { a.v += p; }
__device__ __forceinline__ void shfl_add(AccF& a, int off) {
  float h = __shfl_xor_sync(0xffffffffu, a.hi, off);
  float l = __shfl_xor_sync(0xffffffffu, a.lo, off);
  a.add_pair(h, l);
}
__device__ __forceinline__ void shfl_add(AccD& a, int off) { a.v += __shfl_xor_sync(0xffffffffu, a.v, off); }

__device__ __forceinline__ void zero_part(float2& p) { p = make_float2(0.f, 0.f); }
__device__ __forceinline__ void zero_part(double& p) { p = 0.0; }

// The grid sums of reduce_blocks: warp w takes sums w, w + NW, ... S at a
// time; lane l adds blocks l, l + 32, ... in order (S x UL loads in flight),
// then a fixed shuffle tree; out(p, total) is called from lane 0.
template <int S, int UL, typename Acc, typename Part, typename Out>
__device__ __forceinline__ void sum_partials(const Part* part, int P, int G, int lane, int warp, Out& out) {
  constexpr int NW = kBlockThreads / 32;
  for (int p0 = warp; p0 < P; p0 += S * NW) {
    Acc s[S];
#pragma unroll
    for (int j = 0; j < S; ++j) s[j].zero();
    for (int b0 = 0; b0 < G; b0 += 32 * UL) {
      Part v[S][UL];
#pragma unroll
      for (int j = 0; j < S; ++j)
#pragma unroll
        for (int u = 0; u < UL; ++u) {
          const int b = b0 + u * 32 + lane, p = p0 + j * NW;
          zero_part(v[j][u]);
          if (b < G && p < P) v[j][u] = __ldcg(&part[(size_t)p * G + b]);
        }
#pragma unroll
      for (int j = 0; j < S; ++j)
#pragma unroll
        for (int u = 0; u < UL; ++u) add_part(s[j], v[j][u]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int j = 0; j < S; ++j) shfl_add(s[j], off);
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < S; ++j)
        if (p0 + j * NW < P) out(p0 + j * NW, s[j].value());
  }
}

// Deterministic sum over the G blocks of a grid of P partial sums:
// part[p * G + b] holds block b's partial of sum p (every block has written
// its own before the call).  The last block to arrive (ticket) sums them
// (sum_partials: two sums per warp at a time with 10 loads per lane each, or
// four with 5 when the grid has at most 160 blocks -- the same additions in
// the same order, the absent blocks' loads being zeros either way).  Returns
// true in that block only.  Must be reached by every block of the grid.
template <typename Acc, typename Part, typename Out>
__device__ __forceinline__ bool reduce_blocks(const Part* part, unsigned int* count, int P, int vb, int G, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ unsigned int ticket;
  (void)vb;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(count, 1u);
  __syncthreads();
  if (ticket != (unsigned int)(G - 1)) return false;
  __threadfence();
  if (G <= 32 * 5)
    sum_partials<4, 5, Acc>(part, P, G, lane, warp, out);
  else
    sum_partials<2, 10, Acc>(part, P, G, lane, warp, out);
  __syncthreads();
  if (threadIdx.x == 0) *count = 0u;
  return true;
}

// Block + grid reduction of ND per-component sums, plus NP more sums kept in
// plain T (sums that only set a tolerance or a choice; fewer registers are
// live at the end of a pass than with float-float pairs): within the warp
// they are added in T, from the block partials on like the others.  Every
// block writes its partial; the grid's partials are summed by
// reduce_blocks, which leaves the totals in tot[ND + NP][kMaxCols] of the
// last block (the NP plain sums after the others).  Returns true in the last
// block only.  Must be reached by every block of the grid.
template <typename T, int LPR, int ND, int NP>
__device__ __forceinline__ bool grid_reduce_plain(typename AccOf<T>::type (&acc)[ND][VecW<T>::W],
                                                  T (&pl)[NP > 0 ? NP : 1][VecW<T>::W], const KArgs<T>& a, int slot,
                                                  double (*tot)[kMaxCols], int vb, int vg) {
  typedef typename AccOf<T>::type Acc;
  typedef typename AccOf<T>::part Part;
  constexpr int VW = VecW<T>::W;
  constexpr int NW = kBlockThreads / 32;
  constexpr int NT = ND + NP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cg = lane % LPR;
#pragma unroll
  for (int off = LPR; off < 32; off <<= 1) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < VW; ++v) shfl_add(acc[d][v], off);
#pragma unroll
    for (int d = 0; d < NP; ++d)
#pragma unroll
      for (int v = 0; v < VW; ++v) pl[d][v] += __shfl_xor_sync(0xffffffffu, pl[d][v], off);
  }
  __shared__ Part red[NT][NW][kMaxCols];
  if (lane < LPR) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < VW; ++v) red[d][warp][cg * VW + v] = to_part(acc[d][v]);
#pragma unroll
    for (int d = 0; d < NP; ++d)
#pragma unroll
      for (int v = 0; v < VW; ++v) red[ND + d][warp][cg * VW + v] = plain_part(pl[d][v]);
  }
  __syncthreads();
  const int G = vg;
  Part* part = reinterpret_cast<Part*>(a.part);
  for (int t = threadIdx.x; t < NT * a.ms; t += kBlockThreads) {
    const int d = t / a.ms, c = t % a.ms;
    Acc s;
    s.zero();
    for (int w = 0; w < NW; ++w) add_part(s, red[d][w][c]);
    part[(size_t)(d * a.ms + c) * G + vb] = to_part(s);
  }
  const int ms = a.ms;
  return reduce_blocks<Acc>(part, &a.ctl->counters[slot], NT * ms, vb, G,
                            [&](int p, double v) { tot[p / ms][p % ms] = v; });
}

// grid_reduce_plain without plain sums.
template <typename T, int LPR, int ND>
__device__ __forceinline__ bool grid_reduce(typename AccOf<T>::type (&acc)[ND][VecW<T>::W],
                                            const KArgs<T>& a, int slot, double (*tot)[kMaxCols], int vb, int vg) {
  T none[1][VecW<T>::W];
  return grid_reduce_plain<T, LPR, ND, 0>(acc, none, a, slot, tot, vb, vg);
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

// Rows of a block: a contiguous range [r0, r1) of ceil(n / gridDim.x) rows.
#define SEG_ROW_SETUP                                                         \
  constexpr int VW = VecW<T>::W;                                              \
  constexpr int NW = kBlockThreads / 32;                                      \
  constexpr int RPW = 32 / LPR;                                               \
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;                 \
  const int rs = lane / LPR, cg = lane % LPR, c0 = cg * VW;                   \
  (void)rs;                                                                   \
  const int rpb = (a.n + vg - 1) / vg;                                        \
  const int r0 = vb * rpb;                                                    \
  const int r1 = min(a.n, r0 + rpb);

// Padded-ELL row of W entries: column indices (-1 = padding) and values.
template <int W>
__device__ __forceinline__ void ld_cols(int (&c)[W], const int* p) {
#pragma unroll
  for (int k = 0; k < W; k += 4) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(p + k));
    c[k] = v.x; c[k + 1] = v.y; c[k + 2] = v.z; c[k + 3] = v.w;
  }
}
template <int W>
__device__ __forceinline__ void ld_vals(float (&c)[W], const float* p) {
#pragma unroll
  for (int k = 0; k < W; k += 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p + k));
    c[k] = v.x; c[k + 1] = v.y; c[k + 2] = v.z; c[k + 3] = v.w;
  }
}
template <int W>
__device__ __forceinline__ void ld_vals(double (&c)[W], const double* p) {
#pragma unroll
  for (int k = 0; k < W; k += 2) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p + k));
    c[k] = v.x; c[k + 1] = v.y;
  }
}

// ------------------------------------------------ TMA bulk-copy pipeline

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Invalidate an mbarrier (all its phases complete, no copy in flight) so that
// its shared memory may hold a new one: a block that runs several pipelines
// (the virtual blocks of a batch) initialises its ring afresh for each.
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (TMA); both addresses 16-byte aligned and
// bytes a multiple of 16; completion is signalled on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bounded wait for the phase `parity` of `bar`: false once limit_ns have
// passed (globaltimer; the state's wait limit, 1 s by default).  Each try may
// suspend the warp for up to kSuspendNs until the phase completes, so a
// waiting warp does not spin on the issue slots that the other warps of the
// SM need.
constexpr unsigned kSuspendNs = 2000;
constexpr unsigned long long kWaitNs = kDefaultWaitNs;  // 1 s
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity, unsigned hint_ns) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Non-blocking probe of the phase `parity` of `bar`.
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long limit_ns) {
  if (limit_ns < kSuspendNs) {
    // a limit shorter than one suspension: non-blocking probes only (a
    // suspended try may outlast the limit by the time the data needs),
    // timed in SM clock cycles, 2 per ns (the global timer may tick only
    // every microsecond, which would let data that takes less than that
    // arrive within any shorter limit)
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    const long long cycles = 2 * (long long)limit_ns;
    for (unsigned n = 0; n < (1u << 26); ++n) {
      if (mbar_test_wait(bar, parity)) return true;
      if (clock64() - t0 > cycles) return false;
    }
    return false;
  }
  if (mbar_try_wait(bar, parity, kSuspendNs)) return true;
  const unsigned long long t0 = global_ns();
  // bounded by time and, as a backstop, by the number of tries
  for (unsigned n = 0; n < (1u << 26); ++n) {
    if (mbar_try_wait(bar, parity, kSuspendNs)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Sources of one staged row group (all pointers to row 0 of their array).
template <typename T, int NVAL, int NVEC>
struct StageSrc {
  const int* ell;
  const T* val[NVAL];
  const T* vec[NVEC];  // rows of ms values
};

constexpr int kPipeStages = 4;  // deepest copy ring of the staged row passes

// Per-warp staging of one group of RPW consecutive rows: the padded-ELL
// indices and NVAL value arrays of the group and the rows of NVEC vectors.
// Every piece is a contiguous slice of global memory, copied by one bulk copy.
template <typename T, int LPR, int W, int NVAL, int NVEC>
struct RowStage {
  typedef T value_t;
  typedef StageSrc<T, NVAL, NVEC> Src;
  static constexpr int RPW = 32 / LPR;
  static constexpr int MS = LPR * VecW<T>::W;  // padded components
  static constexpr unsigned kColBytes = RPW * W * 4;
  static constexpr unsigned kValBytes = RPW * W * sizeof(T);
  static constexpr unsigned kVecBytes = RPW * MS * sizeof(T);  // = 512
  static constexpr int kNvec = NVEC;
  static constexpr unsigned kBytes = kColBytes + NVAL * kValBytes + NVEC * kVecBytes;
  // stages of each warp's copy ring (up to kStages - 1 row groups in flight
  // while one is consumed): as many as fit 64 KiB per block, 2 .. kPipeStages
  static constexpr int kStages =
      (int)(65536u / ((kBlockThreads / 32) * kBytes)) < 2
          ? 2
          : ((int)(65536u / ((kBlockThreads / 32) * kBytes)) > kPipeStages
                 ? kPipeStages
                 : (int)(65536u / ((kBlockThreads / 32) * kBytes)));
  static_assert(kColBytes % 16 == 0 && kValBytes % 16 == 0 && kVecBytes % 16 == 0, "16-byte pieces");

  unsigned char* base;
  __device__ __forceinline__ const int* cols() const { return reinterpret_cast<const int*>(base); }
  __device__ __forceinline__ const T* vals(int k) const {
    return reinterpret_cast<const T*>(base + kColBytes + k * kValBytes);
  }
  __device__ __forceinline__ const T* vec(int k) const {
    return reinterpret_cast<const T*>(base + kColBytes + NVAL * kValBytes + k * kVecBytes);
  }
  // lane 0 only: copy rows [row0, row0 + nr) of the sources into this stage
  __device__ __forceinline__ void issue(unsigned long long* bar, int row0, int nr, const Src& src) const {
    const unsigned ncb = nr * W * 4, nvb = nr * W * sizeof(T), nrb = nr * MS * sizeof(T);
    mbar_expect_tx(bar, ncb + NVAL * nvb + NVEC * nrb);
    bulk_g2s(base, src.ell + (size_t)row0 * W, ncb, bar);
#pragma unroll
    for (int k = 0; k < NVAL; ++k)
      bulk_g2s(base + kColBytes + k * kValBytes, src.val[k] + (size_t)row0 * W, nvb, bar);
#pragma unroll
    for (int k = 0; k < NVEC; ++k)
      bulk_g2s(base + kColBytes + NVAL * kValBytes + k * kVecBytes, src.vec[k] + (size_t)row0 * MS, nrb, bar);
  }
};

template <typename Stage>
constexpr unsigned row_stage_smem() {
  return (kBlockThreads / 32) * Stage::kStages * Stage::kBytes;
}

// Reads VW values of this lane from a staged row (shared memory).
__device__ __forceinline__ void lds(float (&d)[4], const float* p) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
}
__device__ __forceinline__ void lds(double (&d)[2], const double* p) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  d[0] = x.x; d[1] = x.y;
}

// Copy one staged padded-ELL row (W indices or values) from shared memory
// into registers with 16-byte loads.
template <int W>
__device__ __forceinline__ void lds_row(int (&d)[W], const int* p) {
#pragma unroll
  for (int k = 0; k < W; k += 4) {
    const int4 v = *reinterpret_cast<const int4*>(p + k);
    d[k] = v.x; d[k + 1] = v.y; d[k + 2] = v.z; d[k + 3] = v.w;
  }
}
template <int W>
__device__ __forceinline__ void lds_row(float (&d)[W], const float* p) {
#pragma unroll
  for (int k = 0; k < W; k += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + k);
    d[k] = v.x; d[k + 1] = v.y; d[k + 2] = v.z; d[k + 3] = v.w;
  }
}
template <int W>
__device__ __forceinline__ void lds_row(double (&d)[W], const double* p) {
#pragma unroll
  for (int k = 0; k < W; k += 2) {
    const double2 v = *reinterpret_cast<const double2*>(p + k);
    d[k] = v.x; d[k + 1] = v.y;
  }
}

// Every hot-path launch is counted once per state (block 0 of the state).
__device__ __forceinline__ void count_launch(DevCtl* ctl, int vb) {
  if (vb == 0 && threadIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
}

// Mark a timed-out wait: the block records the error and halts the run.
__device__ __forceinline__ void report_timeout(DevCtl* ctl) {
  atomicOr(&ctl->status, 4);
  atomicExch(&ctl->halted, 2);
}

// Row groups (RPW consecutive rows) of one block of the staged passes.  The
// mesh's groups are cut into chunks of kChunkGroups groups dealt round-robin
// to the blocks (chunk c to block c mod G), so that every block gets rows
// from all over the mesh: the cost of a row depends on where it lies (the
// locality of its neighbours), and contiguous ranges per block left some
// blocks 10% slower than the median.  Local group k of block vb starts at
// row row0(k).
constexpr int kChunkGroups = 32;
struct GroupMap {
  int n, rpw, vb, vg, ngroups;
  __device__ __forceinline__ int row0(int k) const {
    return ((vb + (k / kChunkGroups) * vg) * kChunkGroups + k % kChunkGroups) * rpw;
  }
};
__device__ __forceinline__ GroupMap group_map(int n, int rpw, int vb, int vg) {
  GroupMap g{n, rpw, vb, vg, 0};
  const int ngt = (n + rpw - 1) / rpw;
  const int nch = (ngt + kChunkGroups - 1) / kChunkGroups;
  if (vb < nch) {
    const int mine = (nch - 1 - vb) / vg + 1;  // chunks vb, vb + vg, ...
    const int last = vb + (mine - 1) * vg;
    g.ngroups = (mine - 1) * kChunkGroups + (last == nch - 1 ? ngt - last * kChunkGroups : kChunkGroups);
  }
  return g;
}

// Warp-level pipeline over the row groups of the block (GroupMap, groups of
// Stage::RPW rows); warp w takes local groups w, w+NW, ...  The copies of the
// warp's next Stage::kStages - 1 groups are in flight while one group is
// processed.  `body(stage, row0, nr)` consumes a landed stage.  Returns false
// if a wait gave up after wait_ns; the copies still in flight are then waited
// for with the default limit kWaitNs, so that none is outstanding when the
// block exits.
template <typename Stage, typename Body>
__device__ __forceinline__ bool row_pipeline(unsigned char* smem_warp, unsigned long long* bars, const GroupMap& gm,
                                             const typename Stage::Src& src, unsigned long long wait_ns, bool stall,
                                             Body body) {
  constexpr int NW = kBlockThreads / 32;
  constexpr int RPW = Stage::RPW;
  constexpr int NS = Stage::kStages;
  static_assert(RPW >= 1 && NS >= 2, "pipeline shape");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ngroups = gm.ngroups;
  const int n = gm.n;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
    mbar_init_fence();
    // the stages may have been read through the generic proxy (an earlier
    // pipeline of this block): order those reads before the copies below
    fence_proxy_async_smem();
  }
  __syncwarp();
  auto stage = [&](int k) {
    Stage sg;
    sg.base = smem_warp + k * Stage::kBytes;
    return sg;
  };
  // prologue: groups 0 .. NS-2 of this warp into stages 0 .. NS-2
  unsigned pending = 0;  // stages with copies in flight (bit mask)
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    const int g = warp + k * NW;
    if (g < ngroups) {
      if (lane == 0) {
        const int row0 = gm.row0(g);
        stage(k).issue(&bars[k], row0, min(RPW, n - row0), src);
      }
      pending |= 1u << k;
    }
  }
  bool ok = true;
  if (stall) {
    // testing aid for the failure path: a bounded wait on a barrier that
    // nothing completes runs out exactly as a wait for data that does not
    // arrive would (the copies issued above land and are drained below)
    __shared__ __align__(8) unsigned long long never[NW];
    if (lane == 0) {
      mbar_init(&never[warp], 1);
      mbar_init_fence();
    }
    __syncwarp();
    ok = __all_sync(0xffffffffu, mbar_wait(&never[warp], 0u, wait_ns));
    __syncwarp();
    if (lane == 0) mbar_inval(&never[warp]);
  }
  unsigned phase = 0;  // bit k: parity of the next completion of stage k
  int s = 0;
  for (int gi = ok ? warp : ngroups; gi < ngroups; gi += NW) {
    // refill the stage consumed in the previous iteration
    const int gn = gi + (NS - 1) * NW;
    const int sn = s == 0 ? NS - 1 : s - 1;
    if (gn < ngroups) {
      if (lane == 0) {
        fence_proxy_async_smem();
        const int row0 = gm.row0(gn);
        stage(sn).issue(&bars[sn], row0, min(RPW, n - row0), src);
      }
      pending |= 1u << sn;
    }
    const bool landed = mbar_wait(&bars[s], (phase >> s) & 1u, wait_ns);
    if (!__all_sync(0xffffffffu, landed)) {
      ok = false;
      break;
    }
    pending &= ~(1u << s);
    phase ^= 1u << s;
    const int row0 = gm.row0(gi);
    body(stage(s), row0, min(RPW, n - row0));
    __syncwarp();
    s = s == NS - 1 ? 0 : s + 1;
  }
  if (!ok) {
    // drain: wait (bounded) for every stage that still has copies in flight
    for (int k = 0; k < NS; ++k)
      if (pending & (1u << k)) mbar_wait(&bars[k], (phase >> k) & 1u, kWaitNs);
  }
  __syncwarp();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NS; ++k) mbar_inval(&bars[k]);
  __syncwarp();
  return ok;
}

template <typename T, int LPR, int W>
using StartStage = RowStage<T, LPR, W, 3, 1>;
// CG pass A in three forms: the first iteration of a solve (kCgFirst: own
// rows of z only), later even iterations (kCgEven: z, p_old, q_old) and odd
// iterations (kCgOdd: also y and p_{j-2} for the two pending solution updates).
constexpr int kCgFirst = 0, kCgEven = 1, kCgOdd = 2;
template <typename T, int LPR, int W, int FORM>
using CgAStage = RowStage<T, LPR, W, 1, FORM == kCgFirst ? 1 : (FORM == kCgOdd ? 5 : 3)>;

// Start pass of the CG solve of step 1, (M + tau K) x = M X, fused with the
// renormalisation of the previous step.  The iterate is x = X + y, with y
// starting at w Y: Y holds this step's correction as the finish pass of the
// previous step predicted it from the last solves' corrections (0 after a
// state is set) and w (per component, 0 or 1) says whether the last start
// pass found the prediction better than none:
//   r0 = M X - (M + tau K)(X + w Y) = -tau K X - w A Y,  z0 = D^-1 r0  -> Z,
// per component  ||X||_M^2, X^T K X, r0.z0  (float-float) and, in float32 per
// thread (they only set the tolerance and the choice of w), ||M X||_2^2 and
// the squared norms of the residuals of both starts, -tau K X and
// -tau K X - A Y.  The next step uses w = 1 where the second was smaller.
template <typename T, int LPR, int W, bool CO = false>
__device__ __forceinline__ void body_start(const KArgs<T>& a, const int vb, const int vg) {
  typedef typename AccOf<T>::type Acc;
  typedef StartStage<T, LPR, W> Stage;
  DevCtl* ctl = a.ctl;
  count_launch(ctl, vb);
  if (state_finished(a, ctl)) return;
  SEG_ROW_SETUP
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  __shared__ __align__(8) unsigned long long bars[NW][kPipeStages];
  const T tau = (T)a.tau;
  const unsigned ms = a.ms;
  Acc acc[3][VW];  // ||X||_M^2, X^T K X, r0.z0
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[d][v].zero();
  T pl[3][VW];  // ||M X||^2, ||-tau K X||^2, ||-tau K X - A Y||^2
  unsigned om = 0;  // bit v: this lane's component c0 + v starts from the predicted correction
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    pl[0][v] = pl[1][v] = pl[2][v] = T(0);
    if (ctl->carry[c0 + v]) om |= 1u << v;
  }
  typename Stage::Src src;
  src.ell = a.ell_col;
  src.val[0] = a.valK;
  src.val[1] = a.valM;
  src.val[2] = a.valA;
  src.vec[0] = a.X;
  const bool ok = row_pipeline<Stage>(
      dyn_smem + warp * Stage::kStages * Stage::kBytes, bars[warp], group_map(a.n, RPW, vb, vg), src, a.wait_ns,
      a.stall_waits != 0, [&](const Stage& sg, int row0, int nr) {
        if (rs >= nr) return;
        const unsigned row = row0 + rs;
        int cols[W];
        T kv[W], mv[W];
        lds_row<W>(cols, sg.cols() + rs * W);
        lds_row<W>(kv, sg.vals(0) + rs * W);
        lds_row<W>(mv, sg.vals(1) + rs * W);
        T x[VW];
        lds(x, sg.vec(0) + rs * ms + c0);
        const T di = __ldg(a.dinv + row);
        // the neighbours' rows of X and Y all in flight at once (padding
        // entries point at the row itself with value 0)
        T xj[W][VW], yj[W][VW];
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const unsigned o = (unsigned)cols[k] * ms + c0;
          ldv<CO>(xj[k], a.X + o);
          ldv<CO>(yj[k], a.Y + o);
        }
        T kx[VW], mx[VW];
#pragma unroll
        for (int v = 0; v < VW; ++v) kx[v] = mx[v] = T(0);
#pragma unroll
        for (int k = 0; k < W; ++k) {
          v_axpy(kx, kv[k], xj[k]);
          v_axpy(mx, mv[k], xj[k]);
        }
        T ay[VW], av[W];
        lds_row<W>(av, sg.vals(2) + rs * W);
#pragma unroll
        for (int v = 0; v < VW; ++v) ay[v] = T(0);
#pragma unroll
        for (int k = 0; k < W; ++k) v_axpy(ay, av[k], yj[k]);
        T ra[VW], rb[VW], r[VW], z[VW];
        v_scale(ra, -tau, kx);
        v_sub(rb, ra, ay);
        v_fma(pl[1], ra, ra, pl[1]);
        v_fma(pl[2], rb, rb, pl[2]);
#pragma unroll
        for (int v = 0; v < VW; ++v) r[v] = (om >> v) & 1u ? rb[v] : ra[v];
        v_scale(z, di, r);
        st(a.Z + (row * ms + c0), z);
        v_add_prods(acc[0], x, mx);
        v_add_prods(acc[1], x, kx);
        v_add_prods(acc[2], r, z);
        v_fma(pl[0], mx, mx, pl[0]);
      });
  if (__syncthreads_or(!ok) && threadIdx.x == 0) report_timeout(ctl);
  __shared__ double tot[6][kMaxCols];
  if (!grid_reduce_plain<T, LPR, 3, 3>(acc, pl, a, kCtrStart, tot, vb, vg)) return;
  int act = 0, bad = 0;
  const int c = threadIdx.x;
  if (a.norm_only) {
    // the normalisation only (reading the state between steps): the solver's
    // scalars, the choice of start and the loop flag keep the values the
    // step before left, so that reading the state does not change the run
    if (c < a.ms) {
      const double n2 = tot[0][c], ukt = tot[1][c];
      const bool real = c < a.m;
      if (real && !(n2 > 0.0 && isfinite(n2) && isfinite(ukt))) bad = 1;
      ctl->n2[c] = n2;
      ctl->inv_n[c] = (real && n2 > 0.0) ? 1.0 / sqrt(n2) : 0.0;
      ctl->lam[c] = (real && n2 > 0.0) ? ukt / n2 : 0.0;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) ctl->status |= 2;
    return;
  }
  if (c < a.ms) {
    const bool used = ctl->carry[c] != 0;
    const double n2 = tot[0][c], ukt = tot[1][c], rz = tot[2][c], bbt = tot[3][c];
    const double rrt = used ? tot[5][c] : tot[4][c];
    const bool real = c < a.m;
    ctl->ysc[c] = used ? 1.0 : 0.0;
    ctl->carry[c] = (real && tot[5][c] < tot[4][c]) ? 1 : 0;
    if (real && !(n2 > 0.0 && isfinite(n2) && isfinite(rrt) && isfinite(ukt))) bad = 1;
    ctl->n2[c] = n2;
    ctl->inv_n[c] = (real && n2 > 0.0) ? 1.0 / sqrt(n2) : 0.0;
    ctl->lam[c] = (real && n2 > 0.0) ? ukt / n2 : 0.0;
    ctl->tol2[c] = a.rtol2 * bbt;
    ctl->rz[c] = rz;
    ctl->rr0[c] = rrt;
    ctl->alpha[0][c] = 0.0;
    ctl->alpha[1][c] = 0.0;
    ctl->beta[c] = 0.0;
    act = (real && !bad && rrt > a.rtol2 * bbt) ? 1 : 0;
    ctl->active[c] = act;
  }
  const int any = __syncthreads_or(act);
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    ctl->it = 0;
    ctl->dir_in_z = 0;
    int cont = (any && !anybad && ctl->halted != 2) ? 1 : 0;
    if (anybad) {
      ctl->status |= 2;
      ctl->halted = 2;
    }
    ctl->cont = cont;
    if (a.set_cond) cudaGraphSetConditional(a.cond, cont);
  }
}

// CG pass A of iteration j (it = j - 1 iterations done):
//   p_j = z_{j-1} + beta p_{j-1}                    (own row)
//   q_j = A p_j = A z_{j-1} + beta q_{j-1}           (q_{j-1} = A p_{j-1} from the
//         previous pass A, own row; only z is gathered from the neighbours)
//   p_j . q_j  (float-float).
// The solution (its correction y, buffer Y) is updated every second
// iteration, two terms at a time (the search directions of the last two
// iterations are both still in the ping-pong buffers): for even j,
// y += alpha_{j-2} p_{j-2} + alpha_{j-1} p_{j-1},
// the same sequence of operations as one lagged update per iteration, with
// one read and write of y saved per two iterations; the finish pass applies
// what is left.  The first iteration of a solve has no previous direction:
// p_1 = z_0 and q_1 = A z_0, and the direction buffers (which hold values of
// the previous solve) are neither staged nor read.  That pass also finds the
// residual norm after the iteration and ends the solve when every component
// has converged, in which case CG pass B has nothing to do (once a run has
// settled, the predicted start leaves one iteration per solve).
// Padded ELL entries point at the row itself with value 0 (no branches).
template <typename T, int LPR, int W, int FORM, bool CO>
__device__ __forceinline__ void body_cg_a_rows(const KArgs<T>& a, const int vb, const int vg, const int it) {
  typedef typename AccOf<T>::type Acc;
  typedef CgAStage<T, LPR, W, FORM> Stage;
  constexpr bool XUP = FORM == kCgOdd;
  DevCtl* ctl = a.ctl;
  SEG_ROW_SETUP
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  __shared__ __align__(8) unsigned long long bars[NW][kPipeStages];
  // read now what the last block needs after the grid sum (written only by
  // other kernels), so that it does not wait for them at the end
  __shared__ double pre_rz[kMaxCols], pre_tol2[kMaxCols], pre_rr0[kMaxCols];
  __shared__ int pre_act[kMaxCols];
  if ((int)threadIdx.x < a.ms) {
    pre_rz[threadIdx.x] = ctl->rz[threadIdx.x];
    pre_act[threadIdx.x] = ctl->active[threadIdx.x];
    pre_tol2[threadIdx.x] = ctl->tol2[threadIdx.x];
    pre_rr0[threadIdx.x] = ctl->rr0[threadIdx.x];
  }
  const T* Pold = (it & 1) ? a.P1 : a.P0;
  T* Pnew = (it & 1) ? a.P0 : a.P1;
  const unsigned ms = a.ms;
  T beta[VW], al1[VW], al2[VW], ysc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    beta[v] = (T)ctl->beta[c0 + v];
    al1[v] = (T)ctl->alpha[it & 1][c0 + v];        // alpha_{j-1}
    al2[v] = (T)ctl->alpha[(it + 1) & 1][c0 + v];  // alpha_{j-2} (this pass overwrites it with alpha_j)
    ysc[v] = it == 1 ? (T)ctl->ysc[c0 + v] : T(1);  // the first update starts from w Y
  }
  // p.q; in the first iteration also r0.q and q.q (r0 = D z0), from which
  // and the start pass's ||r0||^2 the last block finds the residual of the
  // iterate after this iteration without CG pass B.  A lane sums its rows'
  // terms of these two in plain T (few registers: the gathers of the
  // neighbour rows keep theirs) and adds the sums to the grid sum at the end.
  constexpr int ND = FORM == kCgFirst ? 3 : 1;
  Acc acc[ND][VW];
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[d][v].zero();
  T rq[VW], qq[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) rq[v] = qq[v] = T(0);
  typename Stage::Src src;
  src.ell = a.ell_col;
  src.val[0] = a.valA;
  src.vec[0] = a.Z;
  if constexpr (FORM != kCgFirst) {
    src.vec[1] = Pold;
    src.vec[2] = a.Q;
  }
  if constexpr (XUP) {
    src.vec[3] = a.Y;
    // still p_{j-2}; in the second iteration (alpha_0 = 0) there is no p_0
    // and the buffer holds the previous solve's last direction: read the
    // fresh p_1 in its place, so that no value of the previous solve enters
    src.vec[4] = it == 1 ? Pold : Pnew;
  }
  const bool ok = row_pipeline<Stage>(
      dyn_smem + warp * Stage::kStages * Stage::kBytes, bars[warp], group_map(a.n, RPW, vb, vg), src, a.wait_ns,
      a.stall_waits != 0, [&](const Stage& sg, int row0, int nr) {
        if (rs >= nr) return;
        const unsigned row = row0 + rs;
        int cols[W];
        T av[W];
        lds_row<W>(cols, sg.cols() + rs * W);
        lds_row<W>(av, sg.vals(0) + rs * W);
        // all neighbour rows of z in flight at once
        T zj[W][VW];
#pragma unroll
        for (int k = 0; k < W; ++k) ldv<CO>(zj[k], a.Z + ((unsigned)cols[k] * ms + c0));
        T zi[VW], pn[VW], q[VW];
        lds(zi, sg.vec(0) + rs * ms + c0);
#pragma unroll
        for (int v = 0; v < VW; ++v) q[v] = T(0);
#pragma unroll
        for (int k = 0; k < W; ++k) v_axpy(q, av[k], zj[k]);
        if constexpr (FORM == kCgFirst) {
#pragma unroll
          for (int v = 0; v < VW; ++v) pn[v] = zi[v];
        } else {
          T po[VW], qo[VW];
          lds(po, sg.vec(1) + rs * ms + c0);
          lds(qo, sg.vec(2) + rs * ms + c0);
          if constexpr (XUP) {
            T x[VW], pp[VW];
            lds(x, sg.vec(3) + rs * ms + c0);
            lds(pp, sg.vec(4) + rs * ms + c0);
            T y0[VW];
#pragma unroll
            for (int v = 0; v < VW; ++v) y0[v] = ysc[v] * x[v];
            v_fma(y0, al2, pp, y0);
            v_fma(x, al1, po, y0);
            st(a.Y + (row * ms + c0), x);
          }
          v_fma(pn, beta, po, zi);
          v_fma(q, beta, qo, q);
        }
        // (p_1 = z_0 stays in Z: CG pass B copies it to P1 if the solve goes on)
        if constexpr (FORM != kCgFirst) st(Pnew + (row * ms + c0), pn);
        st(a.Q + (row * ms + c0), q);
        v_add_prods(acc[0], pn, q);
        if constexpr (FORM == kCgFirst) {
          T r0[VW];
          v_scale(r0, __ldg(a.diagA + row), zi);
          v_fma(rq, r0, q, rq);
          v_fma(qq, q, q, qq);
        }
      });
  if constexpr (FORM == kCgFirst) {
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      acc[1 % ND][v].add_val(rq[v]);
      acc[2 % ND][v].add_val(qq[v]);
    }
  }
  if (__syncthreads_or(!ok) && threadIdx.x == 0) report_timeout(ctl);
  __shared__ double tot[ND][kMaxCols];
  if (!grid_reduce<T, LPR, ND>(acc, a, kCtrCgA, tot, vb, vg)) return;
  const int c = threadIdx.x;
  int open = 0;
  if (c < a.ms) {
    const double pq = tot[0][c];
    const double al = (pre_act[c] && pq > 0.0) ? pre_rz[c] / pq : 0.0;
    ctl->alpha[(it + 1) & 1][c] = al;
    if constexpr (FORM == kCgFirst) {
      // ||r1||^2 = ||r0 - alpha q||^2 = r0.r0 - 2 alpha r0.q + alpha^2 q.q.
      // The lanes' plain sums of a few dozen rows are accurate to well
      // within 1e-4 (float) or 1e-10 (double) of sum |terms|, and
      // 2 |alpha r0.q| <= r0.r0 + alpha^2 q.q, so that margin times
      // (r0.r0 + alpha^2 q.q) bounds the rounding of the difference: a
      // component within it of its tolerance is left to CG pass B
      const double rr0 = pre_rr0[c], qqs = tot[2 % ND][c];
      const double r1sq = rr0 - 2.0 * al * tot[1 % ND][c] + al * al * qqs;
      const double margin = (sizeof(T) == 4 ? 1e-4 : 1e-10) * (rr0 + al * al * qqs);
      open = (pre_act[c] && !(r1sq + margin <= pre_tol2[c])) ? 1 : 0;
    }
  }
  if constexpr (FORM == kCgFirst) {
    // every component converged in this first iteration: the solve ends here
    // and CG pass B (residual update, r.z, beta) has nothing to do.  The loop
    // flag is left to pass B, which returns at once and clears it: a batched
    // pass A maps its blocks to the members from their flags as its blocks
    // start, so no flag may change while it runs.  (Timing runs repeat the
    // pass on the same data and leave the counters alone.)
    if (!a.force && !__syncthreads_or(open)) {
      if (c < a.ms) ctl->active[c] = 0;
      if (threadIdx.x == 0) {
        ctl->it = 1;
        ctl->dir_in_z = 1;
        if (a.set_cond) cudaGraphSetConditional(a.cond, 0);
      }
    }
  }
}

template <typename T, int LPR, int W, bool CO = false>
__device__ __forceinline__ void body_cg_a(const KArgs<T>& a, const int vb, const int vg) {
  DevCtl* ctl = a.ctl;
  count_launch(ctl, vb);
  if (state_finished(a, ctl)) return;
  if (!ctl->cont && !a.force) return;  // this instance's CG loop has ended (timing runs: force)
  const int it = ctl->it;
  if (it == 0)
    body_cg_a_rows<T, LPR, W, kCgFirst, CO>(a, vb, vg, it);
  else if (it & 1)
    body_cg_a_rows<T, LPR, W, kCgOdd, CO>(a, vb, vg, it);
  else
    body_cg_a_rows<T, LPR, W, kCgEven, CO>(a, vb, vg, it);
}

// The Sec. 2.2 stop rule at a check: the change of the total energy since
// the previous check below energy_tol (absolute, the paper's form) or, if
// energy_rtol > 0, at most energy_rtol times the energy (relative).
template <typename T>
__device__ __forceinline__ bool stop_rule_met(const KArgs<T>& a, double total, const DevCtl* ctl) {
  if (!ctl->have_prev) return false;
  const double d = fabs(total - ctl->e_prev);
  return (a.energy_tol >= 0.0 && d < a.energy_tol) || (a.energy_rtol > 0.0 && d <= a.energy_rtol * fabs(total));
}

// Per-component coupling integral on one flat triangle: with a = (u_i at the
// 3 corners) and B = sum_{j != i} a_j a_j^T the barycentric moments give
//   int_T (a.lam)^2 (lam^T B lam) = |T|/360 [ (s^2 + |a|^2)(1^T B 1 + tr B)
//        + 4 s a^T B 1 + 2 a^T B a + 4 (a o a)^T B 1 + 4 s a^T diag(B)
//        + 6 (a o a)^T diag(B) ],   s = a_0 + a_1 + a_2.
template <typename T>
__device__ __forceinline__ T tri_coupling(T a0, T a1, T a2, T e00, T e11, T e22, T e01, T e02, T e12) {
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
  return (s * s + aa) * (SB + trB) + T(4) * s * aB1 + T(2) * aBa + T(4) * a2B1 + T(4) * s * dBa + T(6) * a2dB;
}

// S_eps and the per-component coupling integrals c_i = int u_i^2 e_i with
// e_i = sum_{j != i} u_j^2, integrated exactly on every flat triangle.  Each
// lane group handles TU triangles per iteration (their corner rows are
// loaded together).
template <typename T, int LPR>
__device__ __forceinline__ void body_energy(const KArgs<T>& a, const int vb, const int vg) {
  typedef typename AccOf<T>::type Acc;
  constexpr int VW = VecW<T>::W;
  constexpr int NW = kBlockThreads / 32;
  constexpr int RPW = 32 / LPR;
  constexpr int TU = 2;
  DevCtl* ctl = a.ctl;
  count_launch(ctl, vb);
  if (state_finished(a, ctl)) return;
  if (!a.force) {
    if (a.check_every <= 0) return;
    if (ctl->step % a.check_every != 0) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rs = lane / LPR, cg = lane % LPR, c0 = cg * VW, lbase = lane - cg;
  const int tpb = (a.ntri + (int)vg - 1) / (int)vg;
  const int t0 = vb * tpb;
  const int t1 = min(a.ntri, t0 + tpb);
  T invn[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) invn[v] = (T)ctl->inv_n[c0 + v];
  Acc acc[1][VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[0][v].zero();
  const T inv360 = T(1) / T(360);
  for (int base = t0 + warp * RPW * TU; base < t1; base += NW * RPW * TU) {
    T u[TU][3][VW];
    T area[TU];
#pragma unroll
    for (int q = 0; q < TU; ++q) {
      const int t = base + q * RPW + rs;
      area[q] = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int v = 0; v < VW; ++v) u[q][k][v] = T(0);
      if (t < t1) {
        const int* tr = a.tri + 3 * (size_t)t;
        const int z0 = __ldg(tr), z1 = __ldg(tr + 1), z2 = __ldg(tr + 2);
        ld_ro(u[q][0], a.X + (size_t)z0 * a.ms + c0);
        ld_ro(u[q][1], a.X + (size_t)z1 * a.ms + c0);
        ld_ro(u[q][2], a.X + (size_t)z2 * a.ms + c0);
        area[q] = __ldg(a.tarea + t);
      }
    }
#pragma unroll
    for (int q = 0; q < TU; ++q) {
      T P[6][VW], E[6][VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const T b0 = u[q][0][v] * invn[v], b1 = u[q][1][v] * invn[v], b2 = u[q][2][v] * invn[v];
        u[q][0][v] = b0;
        u[q][1][v] = b1;
        u[q][2][v] = b2;
        P[0][v] = b0 * b0;
        P[1][v] = b1 * b1;
        P[2][v] = b2 * b2;
        P[3][v] = b0 * b1;
        P[4][v] = b0 * b2;
        P[5][v] = b1 * b2;
      }
      row_exclusive<T, LPR, 6>(P, E, lbase, cg);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const T F = tri_coupling<T>(u[q][0][v], u[q][1][v], u[q][2][v], E[0][v], E[1][v], E[2][v], E[3][v],
                                    E[4][v], E[5][v]);
        acc[0][v].add_val(area[q] * inv360 * F);
      }
    }
  }
  __shared__ double tot[1][kMaxCols];
  if (!grid_reduce<T, LPR, 1>(acc, a, kCtrEnergy, tot, vb, vg)) return;
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
        if (stop_rule_met(a, total, ctl)) {
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

// Block + grid reduction of one float-float (or double) scalar per thread,
// same ticket protocol as grid_reduce; the total lands in *tot of the last
// block, which returns true.
template <typename T>
__device__ __forceinline__ bool grid_reduce_scalar(typename AccOf<T>::type acc, DevCtl* ctl, void* partv, int slot,
                                                   double* tot, int vb, int vg) {
  typedef typename AccOf<T>::type Acc;
  typedef typename AccOf<T>::part Part;
  constexpr int NW = kBlockThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) shfl_add(acc, off);
  __shared__ Part red[NW];
  if (lane == 0) red[warp] = to_part(acc);
  __syncthreads();
  Part* part = reinterpret_cast<Part*>(partv);
  if (threadIdx.x == 0) {
    Acc s;
    s.zero();
    for (int w = 0; w < NW; ++w) add_part(s, red[w]);
    part[vb] = to_part(s);
  }
  return reduce_blocks<Acc>(part, &ctl->counters[slot], 1, vb, vg,
                            [&](int, double v) { *tot = v; });
}

// Symmetric 6-point rule of degree 4 on a triangle (two orbits of points
// with barycentric coordinates (a, a, 1 - 2a)); weights sum to 1, so
// int_T f = |T| sum_q w_q f(q) for every polynomial of degree <= 4.  The
// constants solve the moment equations of the barycentric monomials.
constexpr double kQuadA1 = 0.4459484909159649;
constexpr double kQuadW1 = 0.22338158967801156;
constexpr double kQuadA2 = 0.0915762135097707;
constexpr double kQuadW2 = 0.10995174365532179;

// The pair sums of the degree-4 rule over the components of one triangle:
// at each of the 6 points q the value of u_i is a*tot + (b - a)*corner
// (b = 1 - 2a, tot the sum of the corner values), and
//   sum[q] = sum_i u_i(q)^2 sum_{j < i} u_j(q)^2   (prefix form).
// Returns sum[0] + sum[1] + sum[2] (first orbit) and sum[3] + sum[4] +
// sum[5] (second orbit).  The float version keeps the two orbits' points at
// the same corner in one packed pair (points 0 and 3, 1 and 4, 2 and 5):
// the same operations in the same order, three pairs instead of six values.
template <int MS, bool CO>
__device__ __forceinline__ void quad_pairs(const double* X, unsigned z0, unsigned z1, unsigned z2,
                                           const double* sinv, double A1, double B1mA1, double A2, double B2mA2,
                                           double& sum1, double& sum2) {
  typedef double T;
  // the rows in 32-byte pieces where they hold whole ones (fewer, wider
  // scattered loads: the pass is bound by the L1's handling of them)
  constexpr int VW = MS % 4 == 0 ? 4 : VecW<T>::W;
  T pre[6], sum[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) pre[q] = sum[q] = T(0);
#pragma unroll
  for (int c = 0; c < MS; c += VW) {
    T u0[VW], u1[VW], u2[VW];
    if constexpr (VW == 4 && CO) {
      ld32(u0, X + (z0 + c));
      ld32(u1, X + (z1 + c));
      ld32(u2, X + (z2 + c));
    } else if constexpr (VW == 4) {
      ld_ro32(u0, X + (z0 + c));
      ld_ro32(u1, X + (z1 + c));
      ld_ro32(u2, X + (z2 + c));
    } else {
      ldv<CO>(u0, X + (z0 + c));
      ldv<CO>(u1, X + (z1 + c));
      ldv<CO>(u2, X + (z2 + c));
    }
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const T s = sinv[c + v];
      const T b0 = u0[v] * s, b1 = u1[v] * s, b2 = u2[v] * s;
      const T tot = b0 + b1 + b2;
      const T o1 = A1 * tot, o2 = A2 * tot;
      T val[6];
      val[0] = fma(B1mA1, b0, o1);
      val[1] = fma(B1mA1, b1, o1);
      val[2] = fma(B1mA1, b2, o1);
      val[3] = fma(B2mA2, b0, o2);
      val[4] = fma(B2mA2, b1, o2);
      val[5] = fma(B2mA2, b2, o2);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const T sq = val[q] * val[q];
        sum[q] = fma(sq, pre[q], sum[q]);
        pre[q] += sq;
      }
    }
  }
  sum1 = sum[0] + sum[1] + sum[2];
  sum2 = sum[3] + sum[4] + sum[5];
}
template <int MS, bool CO>
__device__ __forceinline__ void quad_pairs(const float* X, unsigned z0, unsigned z1, unsigned z2, const float* sinv,
                                             float A1, float B1mA1, float A2, float B2mA2, float& sum1, float& sum2) {
  const float2 A = f2(A1, A2), B = f2(B1mA1, B2mA2);
  // the rows in 32-byte pieces where they hold whole ones (see above)
  constexpr int CW = MS % 8 == 0 ? 8 : 4;
  float2 pre[3], sum[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) pre[k] = sum[k] = f2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < MS; c += CW) {
    float u0[CW], u1[CW], u2[CW];
    if constexpr (CW == 8 && CO) {
      ld32(u0, X + (z0 + c));
      ld32(u1, X + (z1 + c));
      ld32(u2, X + (z2 + c));
    } else if constexpr (CW == 8) {
      ld_ro32(u0, X + (z0 + c));
      ld_ro32(u1, X + (z1 + c));
      ld_ro32(u2, X + (z2 + c));
    } else {
      ldv<CO>(u0, X + (z0 + c));
      ldv<CO>(u1, X + (z1 + c));
      ldv<CO>(u2, X + (z2 + c));
    }
#pragma unroll
    for (int v = 0; v < CW; ++v) {
      const float s = sinv[c + v];
      const float b0 = u0[v] * s, b1 = u1[v] * s, b2 = u2[v] * s;
      const float tot = b0 + b1 + b2;
      const float2 o = __fmul2_rn(A, f2(tot, tot));
      float2 val[3];
      val[0] = __ffma2_rn(B, f2(b0, b0), o);
      val[1] = __ffma2_rn(B, f2(b1, b1), o);
      val[2] = __ffma2_rn(B, f2(b2, b2), o);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 sq = __fmul2_rn(val[k], val[k]);
        sum[k] = __ffma2_rn(sq, pre[k], sum[k]);
        pre[k] = __fadd2_rn(pre[k], sq);
      }
    }
  }
  const float2 t = __fadd2_rn(__fadd2_rn(sum[0], sum[1]), sum[2]);
  sum1 = t.x;
  sum2 = t.y;
}

// S_eps of the normalised state for the stop rule (and seg_energy): one
// thread per triangle, the degree-4 rule, and the pair sum in prefix form
//   sum_{i != j} u_i^2 u_j^2 = 2 sum_i u_i^2 sum_{j < i} u_j^2
// (non-negative terms only, no cancellation).  Components are visited in
// chunks of VW so that only one chunk of the three corner rows is live.
template <typename T, int LPR, bool CO = false>
__device__ __forceinline__ void body_energy_check(const KArgs<T>& a, const int vb, const int vg) {
  typedef typename AccOf<T>::type Acc;
  constexpr int VW = VecW<T>::W;
  constexpr int MS = LPR * VW;
  DevCtl* ctl = a.ctl;
  count_launch(ctl, vb);
  if (state_finished(a, ctl)) return;
  if (!a.force) {
    if (a.check_every <= 0) return;
    if (ctl->step % a.check_every != 0) return;
  }
  __shared__ T sinv[MS];
  if (threadIdx.x < MS) sinv[threadIdx.x] = (T)ctl->inv_n[threadIdx.x];
  __syncthreads();
  const T A1 = (T)kQuadA1, B1mA1 = (T)(1.0 - 3.0 * kQuadA1), W1 = (T)kQuadW1;
  const T A2 = (T)kQuadA2, B2mA2 = (T)(1.0 - 3.0 * kQuadA2), W2 = (T)kQuadW2;
  const unsigned ms = MS;
  Acc acc;
  acc.zero();
  for (int t = vb * kBlockThreads + threadIdx.x; t < a.ntri; t += vg * kBlockThreads) {
    const int* tr = a.tri + 3 * (size_t)t;
    const unsigned z0 = __ldg(tr) * ms, z1 = __ldg(tr + 1) * ms, z2 = __ldg(tr + 2) * ms;
    const T area = __ldg(a.tarea + t);
    T sum1, sum2;
    quad_pairs<MS, CO>(a.X, z0, z1, z2, sinv, A1, B1mA1, A2, B2mA2, sum1, sum2);
    const T st = T(2) * area * (W1 * sum1 + W2 * sum2);
    acc.add_val(st);
  }
  __shared__ double tot;
  if (!grid_reduce_scalar<T>(acc, ctl, a.part, kCtrEnergy, &tot, vb, vg)) return;
  if (threadIdx.x == 0) {
    double D = 0.0;
    for (int c = 0; c < a.m; ++c) D += ctl->lam[c];
    const double S = tot * a.inv_eps2;
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
        if (stop_rule_met(a, total, ctl)) {
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

// Streaming passes handle RU rows per lane group per iteration, loading all
// of them before any arithmetic so that enough bytes are in flight per SM.
constexpr int kStreamRows = 4;

// CG pass B of iteration j: z_j = z_{j-1} - alpha_j D^-1 q_j (= D^-1 r_j),
// r_j = D z_j; per component r_j.z_j (float-float) and ||r_j||^2 (float32
// per thread, tolerance only); convergence test and beta for iteration j+1.
template <typename T, int LPR, bool CO = false>
__device__ __forceinline__ void body_cg_b(const KArgs<T>& a, const int vb, const int vg) {
  typedef typename AccOf<T>::type Acc;
  constexpr int RU = kStreamRows;
  DevCtl* ctl = a.ctl;
  count_launch(ctl, vb);
  if (state_finished(a, ctl)) {
    // a kernel of this iteration halted the run: end the CG loop
    if (a.set_cond && vb == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
    return;
  }
  if (!ctl->cont && !a.force) return;  // this instance's CG loop has ended (timing runs: force)
  if (ctl->dir_in_z && !a.force) {
    // the solve ended in its first CG pass A: end the loop
    if (vb == 0 && threadIdx.x == 0) {
      ctl->cont = 0;
      if (a.set_cond) cudaGraphSetConditional(a.cond, 0);
    }
    return;
  }
  SEG_ROW_SETUP
  const int it = ctl->it;
  // read now what the last block needs after the grid sum
  __shared__ double pre_rz[kMaxCols], pre_tol2[kMaxCols];
  __shared__ int pre_act[kMaxCols];
  if ((int)threadIdx.x < a.ms) {
    pre_rz[threadIdx.x] = ctl->rz[threadIdx.x];
    pre_tol2[threadIdx.x] = ctl->tol2[threadIdx.x];
    pre_act[threadIdx.x] = ctl->active[threadIdx.x];
  }
  const unsigned ms = a.ms;
  T nal[VW];  // -alpha_j
#pragma unroll
  for (int v = 0; v < VW; ++v) nal[v] = -(T)ctl->alpha[(it + 1) & 1][c0 + v];
  Acc acc[2][VW];
#pragma unroll
  for (int d = 0; d < 2; ++d)
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[d][v].zero();
  T rr[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) rr[v] = T(0);
  for (int base = r0 + warp * RPW * RU; base < r1; base += NW * RPW * RU) {
    T z[RU][VW], q[RU][VW], di[RU], dg[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const unsigned row = base + u * RPW + rs;
      if ((int)row < r1) {
        ld(z[u], a.Z + (row * ms + c0));
        ldv<CO>(q[u], a.Q + (row * ms + c0));
        di[u] = __ldg(a.dinv + row);
        dg[u] = __ldg(a.diagA + row);
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const unsigned row = base + u * RPW + rs;
      if ((int)row < r1) {
        if (it == 0) st(a.P1 + (row * ms + c0), z[u]);  // p_1 = z_0, left in Z by the first pass A
        T r[VW], dq[VW];
        v_scale(dq, di[u], q[u]);
        v_fma(z[u], nal, dq, z[u]);
        v_scale(r, dg[u], z[u]);
        st(a.Z + (row * ms + c0), z[u]);
        v_add_prods(acc[0], r, z[u]);
        v_fma(rr, r, r, rr);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[1][v].add_val(rr[v]);
  __shared__ double tot[2][kMaxCols];
  if (!grid_reduce<T, LPR, 2>(acc, a, kCtrCgB, tot, vb, vg)) return;
  int act = 0, bad = 0;
  const int c = threadIdx.x;
  if (c < a.ms) {
    const double rzn = tot[0][c], rrn = tot[1][c];
    act = pre_act[c];
    if (c < a.m && !(isfinite(rzn) && isfinite(rrn))) bad = 1;
    if (act && rrn <= pre_tol2[c]) act = 0;
    const double rzo = pre_rz[c];
    ctl->beta[c] = rzo > 0.0 ? rzn / rzo : 0.0;
    ctl->rz[c] = rzn;
    ctl->active[c] = act;
  }
  const int any = __syncthreads_or(act);
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    const int it1 = it + 1;
    ctl->it = a.force ? it : it1;  // (timing runs repeat the same iteration)
    int cont = (any && it1 < a.maxit && ctl->halted != 2) ? 1 : 0;
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

// The solve's result x = X + y_k with the CG updates of y not yet applied
// (lagged from the last iterations; apply_x, else x = X), then the exact
// solution of the nodal ODE of step 2 (Jacobi form):
//   u~ = x * inv_n,  u^_i = u~_i exp(-(2 tau/eps^2) sum_{j != i} u~_j^2)  -> X.
// With apply_x the next solve's initial correction is predicted by
// extrapolation of the last corrections: quadratic for float data,
// Y = 3 y_k - 3 y_{k-1} + y_{k-2}, with H0, H1 keeping the last two (step k
// reads y_{k-1} from H[(k+1) % 2] and y_{k-2} from H[k % 2], then writes y_k
// over the latter); cubic for double data, Y = 4 y_k - 6 y_{k-1} + 4 y_{k-2}
// - y_{k-3}, with H0, H1, H2 keeping the last three (step j's in H[j % 3]).
// (In float32 the cubic rule's amplification of rounding outweighs its
// better prediction.)  Any initial guess gives the same solution to the
// solve's tolerance.
// The solution updates CG pass A has not applied yet: alpha_k p_k (none if
// k = 0), and alpha_{k-1} p_{k-1} before it (TWO) when the iteration count k
// is odd and at least 3.
template <typename T, int LPR, int RU, bool TWO, bool CO>
__device__ __forceinline__ void body_finish_rows(const KArgs<T>& a, const int vb, const int vg, const int it) {
  DevCtl* ctl = a.ctl;
  SEG_ROW_SETUP
  const int lbase = lane - cg;
  // the last direction; after a solve of one iteration that ended in CG
  // pass A it is z_0, still in Z
  const T* P = (it == 1 && ctl->dir_in_z) ? a.Z : ((it & 1) ? a.P1 : a.P0);
  const T* P2 = (it & 1) ? a.P0 : a.P1;
  // history slots of the corrections: two (quadratic prediction) for
  // float, three (cubic) for double; step j's correction is in H[j % NH]
  constexpr int NH = sizeof(T) == 8 ? 3 : 2;
  const int kh = (int)(ctl->step % NH);
  T* const Hm1 = kh == 0 ? (NH == 3 ? a.H2 : a.H1) : (kh == 1 ? a.H0 : a.H1);  // y_{k-1}
  T* const Hm2 = NH == 3 ? (kh == 0 ? a.H1 : (kh == 1 ? a.H2 : a.H0)) : (kh == 0 ? a.H0 : a.H1);  // y_{k-2}
  T* const Hm3 = NH == 3 ? (kh == 0 ? a.H0 : (kh == 1 ? a.H1 : a.H2)) : Hm2;  // y_{k-3} (cubic only)
  T* const Hnew = NH == 3 ? Hm3 : Hm2;  // the oldest, replaced by y_k
  constexpr bool two = TWO;
  const unsigned ms = a.ms;
  T al[VW], al2[VW], invn[VW], ysc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    al[v] = a.apply_x ? (T)ctl->alpha[it & 1][c0 + v] : T(0);
    al2[v] = two ? (T)ctl->alpha[(it + 1) & 1][c0 + v] : T(0);
    invn[v] = (T)ctl->inv_n[c0 + v];
    ysc[v] = it < 2 ? (T)ctl->ysc[c0 + v] : T(1);  // no update of Y yet in this solve: y = w Y
  }
  const T mcoef = -(T)a.coef;
  for (int base = r0 + warp * RPW * RU; base < r1; base += NW * RPW * RU) {
    T x[RU][VW], y[RU][VW], h1[RU][VW], h2[RU][VW], h3[NH == 3 ? RU : 1][VW], p[RU][VW],
        p2[TWO ? RU : 1][VW];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const unsigned row = base + u * RPW + rs;
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        x[u][v] = y[u][v] = h1[u][v] = h2[u][v] = p[u][v] = T(0);
        h3[NH == 3 ? u : 0][v] = T(0);
        if (two) p2[u][v] = T(0);
      }
      if ((int)row < r1) {
        ld(x[u], a.X + (row * ms + c0));
        if (a.apply_x) {
          ld(y[u], a.Y + (row * ms + c0));
          ld(h1[u], Hm1 + (row * ms + c0));
          ld(h2[u], Hm2 + (row * ms + c0));
          if (NH == 3) ld(h3[NH == 3 ? u : 0], Hm3 + (row * ms + c0));
          if (it > 0) ldv<CO>(p[u], P + (row * ms + c0));
        }
        if (two) ldv<CO>(p2[TWO ? u : 0], P2 + (row * ms + c0));
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const unsigned row = base + u * RPW + rs;
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        // (after one iteration there is no alpha_0 term, after none no
        // update: the direction buffers then hold the previous solve's)
        y[u][v] *= ysc[v];
        if (two) y[u][v] = fma(al2[v], p2[TWO ? u : 0][v], y[u][v]);
        if (it > 0) y[u][v] = fma(al[v], p[u][v], y[u][v]);  // the solve's correction y_k
        x[u][v] += y[u][v];
      }
      if (a.apply_x && (int)row < r1) {
        // the next solve's predicted correction, quadratic 3 (y_k - y_{k-1}) + y_{k-2}
        // or cubic 4 (y_k + y_{k-2}) - 6 y_{k-1} - y_{k-3}; y_k kept
        T g[VW];
#pragma unroll
        for (int v = 0; v < VW; ++v)
          g[v] = NH == 3 ? fma(T(4), y[u][v] + h2[u][v], fma(T(-6), h1[u][v], -h3[NH == 3 ? u : 0][v]))
                         : fma(T(3), y[u][v] - h1[u][v], h2[u][v]);
        st(a.Y + (row * ms + c0), g);
        st(Hnew + (row * ms + c0), y[u]);
      }
      if (a.apply_ode) {
        T sq[1][VW], ex[1][VW], ut[VW];
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          ut[v] = x[u][v] * invn[v];
          sq[0][v] = ut[v] * ut[v];
        }
        row_exclusive<T, LPR, 1>(sq, ex, lbase, cg);
#pragma unroll
        for (int v = 0; v < VW; ++v) x[u][v] = ut[v] * t_exp(mcoef * ex[0][v]);
      }
      if ((int)row < r1) st(a.X + (row * ms + c0), x[u]);
    }
  }
}

template <typename T, int LPR, bool CO = false>
__device__ __forceinline__ void body_finish(const KArgs<T>& a, const int vb, const int vg) {
  DevCtl* ctl = a.ctl;
  count_launch(ctl, vb);
  if (state_finished(a, ctl)) return;
  const int it = ctl->it;
  // rows in flight per lane group: fewer where more vectors are read per row
  // (the registers of 2 resident blocks per SM)
  constexpr int RU = sizeof(T) == 8 ? kStreamRows / 2 : kStreamRows - 1;
  // two pending updates after an odd count of 3 or more iterations (after
  // one, the second term would be alpha_0 p_0: there is none)
  if (a.apply_x && (it & 1) && it > 1)
    body_finish_rows<T, LPR, RU - 1, true, CO>(a, vb, vg, it);
  else
    body_finish_rows<T, LPR, RU, false, CO>(a, vb, vg, it);
  if (a.count_step) {
    // the step is counted by the last block to finish, after every block has
    // passed its own state_finished() test (a block that started after an
    // early increment would otherwise see the step limit and skip its rows)
    __shared__ unsigned int fin_ticket;
    __syncthreads();
    if (threadIdx.x == 0) fin_ticket = atomicAdd(&ctl->counters[kCtrFinish], 1u);
    __syncthreads();
    if (threadIdx.x == 0 && fin_ticket == (unsigned int)(vg - 1)) {
      ctl->counters[kCtrFinish] = 0u;
      ctl->step += 1;
      ctl->cg_last = it;
      ctl->cg_total += it;
      if (it > ctl->cg_max) ctl->cg_max = it;
    }
  }
}


// ------------------------------------------------- kernels and batch kernels

// One launch per pass: the single-instance kernels run a body over the whole
// grid; the batch kernels run the virtual blocks of the members taking part
// (BatchArgs) on their physical blocks, block b taking virtual blocks b,
// b + gridDim.x, ...  Members of CG pass A are those whose loop flag is set
// (written before the launch by the previous pass B, the start pass or the
// energy check); physical block 0 records them for pass B, whose own last
// blocks rewrite the flags during its launch.  The other passes take every
// member (a member that has stopped returns at once).
template <typename T, typename Body>
__device__ __forceinline__ void run_batch(const BatchArgs<T>& b, Body body) {
  __shared__ int vstart[kMaxBatch + 1];
  if (threadIdx.x < 32) {
    // lane i decides for member i (all members' flags read at once), then an
    // exclusive scan of the members' virtual blocks over the warp
    const int i = threadIdx.x;
    int take = 0;
    if (i < b.ninst) {
      take = 1;
      if (b.map == kMapCgA) {
        const KArgs<T>& a = b.tab[i];
        take = (a.ctl->cont && !state_finished(a, a.ctl)) ? 1 : 0;
        if (blockIdx.x == 0) b.amap[i] = take;
      } else if (b.map == kMapCgB) {
        take = b.amap[i];
      }
    }
    const int cnt = take ? b.vg[i < b.ninst ? i : 0] : 0;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (i >= off) incl += y;
    }
    if (i < b.ninst) vstart[i] = incl - cnt;
    if (i == b.ninst - 1) vstart[b.ninst] = incl;
  }
  __syncthreads();
  const int total = vstart[b.ninst];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    int i = 0;
    while (i + 1 < b.ninst && v >= vstart[i + 1]) ++i;
    body(b.tab[i], v - vstart[i], b.vg[i]);
    __syncthreads();  // the next virtual block reuses the shared memory
  }
}

#define SEG_DEFINE_PASS(NAME, MINB, TPL, ...)                                                           \
  TPL __global__ void __launch_bounds__(kBlockThreads, MINB) k_##NAME(const KArgs<T> a) {           \
    body_##NAME<__VA_ARGS__>(a, blockIdx.x, gridDim.x);                                             \
  }                                                                                                 \
  TPL __global__ void __launch_bounds__(kBlockThreads, MINB) kb_##NAME(const BatchArgs<T> b) {         \
    run_batch(b, [&](const KArgs<T>& a, int vb, int vg) { body_##NAME<__VA_ARGS__>(a, vb, vg); });   \
  }

#define SEG_TPL_W template <typename T, int LPR, int W>
#define SEG_TPL template <typename T, int LPR>
// The start pass (three sparse products and three float-float sums per row)
// is compiled for one resident block per SM, so that it does not spill.
SEG_DEFINE_PASS(start, kStartBlocksPerSM, SEG_TPL_W, T, LPR, W)
SEG_DEFINE_PASS(cg_a, kRowBlocksPerSM, SEG_TPL_W, T, LPR, W)
SEG_DEFINE_PASS(cg_b, kRowBlocksPerSM, SEG_TPL, T, LPR)
SEG_DEFINE_PASS(finish, kRowBlocksPerSM, SEG_TPL, T, LPR)
SEG_DEFINE_PASS(energy, 2, SEG_TPL, T, LPR)
SEG_DEFINE_PASS(energy_check, kTriBlocksPerSM, SEG_TPL, T, LPR)
#undef SEG_TPL
#undef SEG_TPL_W
#undef SEG_DEFINE_PASS

// Condition of a batch's CG loop (after a CG pass A): continue while any
// instance needs a pass B, i.e. is iterating and did not end its solve in
// its first pass A.
template <typename T>
__global__ void k_batch_vote(const BatchArgs<T> b) {
  int go = 0;
  if ((int)threadIdx.x < b.ninst) {
    const KArgs<T>& a = b.tab[threadIdx.x];
    go = (a.ctl->cont && !a.ctl->dir_in_z && !state_finished(a, a.ctl)) ? 1 : 0;
  }
  const int any = __syncthreads_or(go);
  if (threadIdx.x == 0) cudaGraphSetConditional(b.cond, any);
}

// ------------------------------------------------ persistent batched steps

__device__ __forceinline__ int vld(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ long long vld(const long long* p) { return *(const volatile long long*)p; }

// state_finished() from the control block as it is now in memory (the last
// block of a barrier reads what other blocks wrote in the phase before).
template <typename T>
__device__ __forceinline__ bool finished_now(const KArgs<T>& a) {
  const int halted = vld(&a.ctl->halted);
  return halted != 0 || (a.max_steps > 0 && vld(&a.ctl->step) >= a.max_steps);
}

enum PersistSync { kSyncPlain = 0, kSyncMapA = 1, kSyncAfterA = 2, kSyncEnd = 3 };

// Grid barrier of a cooperative launch.  Thread 0 of each block arrives on a
// counter; in the block that arrives last, warp 0 computes the decisions of
// `kind` from the members' control blocks (lane i for member i, all loads
// in one round), then thread 0 releases the others by advancing the
// generation.  Waits are bounded by wait_ns: a wait that runs out (or sees
// that another block's did) marks every member halted with a timeout and
// returns false, and the kernel returns.  After the barrier the bulk-copy
// engine may read what the phase before wrote (proxy fence).
template <typename T>
__device__ __noinline__ bool persist_sync(const PersistArgs<T>& p, const int kind) {
  PersistCtl* pc = p.pc;
  __shared__ int last_s, ok_s;
  __shared__ unsigned gen_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = *(volatile unsigned*)&pc->gen;
    __threadfence();
    const int last = atomicAdd(&pc->count, 1u) == gridDim.x - 1;
    if (last) pc->count = 0u;
    last_s = last;
    gen_s = g;
    ok_s = 1;
  }
  __syncthreads();
  if (last_s) {
    if (threadIdx.x < 32) {
      const int i = threadIdx.x;
      int go = 0, act = 0;
      if (i < p.ninst) {
        const KArgs<T>& a = p.tab[i];
        const bool fin = finished_now(a);
        act = fin ? 0 : 1;
        if (kind == kSyncMapA) {
          *(volatile int*)&pc->map_a[i] = (vld(&a.ctl->cont) && !fin) ? 1 : 0;
        } else if (kind == kSyncAfterA) {
          *(volatile int*)&pc->map_b[i] = vld(&pc->map_a[i]);
          go = (vld(&a.ctl->cont) && !vld(&a.ctl->dir_in_z) && !fin) ? 1 : 0;
        }
      }
      go = __any_sync(0xffffffffu, go);
      act = __any_sync(0xffffffffu, act);
      if (i == 0) {
        if (kind == kSyncAfterA) *(volatile int*)&pc->go = go;
        if (kind == kSyncEnd) *(volatile int*)&pc->active = act;
        __threadfence();
        atomicExch(&pc->gen, gen_s + 1u);
      }
    }
  } else if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    int ok = 1;
    for (unsigned n = 0;; ++n) {
      if (*(volatile unsigned*)&pc->gen != gen_s) break;
      if ((n & 63u) == 63u && (vld(&pc->status) != 0 || global_ns() - t0 > p.wait_ns || n > (1u << 30))) {
        ok = 0;
        break;
      }
      if (n > 4096) __nanosleep(32);
    }
    __threadfence();
    ok_s = ok;
  }
  if (threadIdx.x == 0) {
    if (!ok_s || vld(&pc->status) != 0) {
      ok_s = 0;
      atomicOr(&pc->status, 1);
      for (int i = 0; i < p.ninst; ++i) report_timeout(p.tab[i].ctl);
    }
  }
  __syncthreads();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return ok_s != 0;
}

// One phase: the virtual blocks of the members taking part (take[i] != 0,
// or all with take == nullptr), block b taking virtual blocks b, b +
// gridDim.x, ... in member order.
template <typename T, typename Body>
__device__ __forceinline__ void persist_phase(const PersistArgs<T>& p, const int* vgs, const int* take, Body body) {
  __shared__ int vstart[kMaxBatch + 1];
  if (threadIdx.x < 32) {
    const int i = threadIdx.x;
    int t = 0;
    if (i < p.ninst) t = take ? vld(take + i) : 1;
    const int cnt = t ? vgs[i < p.ninst ? i : 0] : 0;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (i >= off) incl += y;
    }
    if (i < p.ninst) vstart[i] = incl - cnt;
    if (i == p.ninst - 1) vstart[p.ninst] = incl;
  }
  __syncthreads();
  const int total = vstart[p.ninst];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    int i = 0;
    while (i + 1 < p.ninst && v >= vstart[i + 1]) ++i;
    body(p.tab[i], v - vstart[i], vgs[i]);
    __syncthreads();  // the next virtual block reuses the shared memory
  }
}

// Up to p.nsteps whole steps of every member (Algorithm 2.2, the same passes
// and the same arithmetic as the step graph; coherent loads for the vectors,
// which earlier phases of the launch write).  Ends early once every member
// has finished (stop rule, step limit or error).
template <typename T, int LPR, int W>
__global__ void __launch_bounds__(kBlockThreads, 1) k_persist(const PersistArgs<T> p) {
  PersistCtl* pc = p.pc;
  for (long long step = 0; step < p.nsteps; ++step) {
    persist_phase(p, p.vg[kPassStart], nullptr,
                  [&](const KArgs<T>& a, int vb, int vg) { body_start<T, LPR, W, true>(a, vb, vg); });
    if (!persist_sync(p, kSyncPlain)) return;
    persist_phase(p, p.vg[4], nullptr,
                  [&](const KArgs<T>& a, int vb, int vg) { body_energy_check<T, LPR, true>(a, vb, vg); });
    if (!persist_sync(p, kSyncMapA)) return;
    persist_phase(p, p.vg[kPassCgA], pc->map_a,
                  [&](const KArgs<T>& a, int vb, int vg) { body_cg_a<T, LPR, W, true>(a, vb, vg); });
    if (!persist_sync(p, kSyncAfterA)) return;
    while (vld(&pc->go)) {
      persist_phase(p, p.vg[kPassCgB], pc->map_b,
                    [&](const KArgs<T>& a, int vb, int vg) { body_cg_b<T, LPR, true>(a, vb, vg); });
      if (!persist_sync(p, kSyncMapA)) return;
      persist_phase(p, p.vg[kPassCgA], pc->map_a,
                    [&](const KArgs<T>& a, int vb, int vg) { body_cg_a<T, LPR, W, true>(a, vb, vg); });
      if (!persist_sync(p, kSyncAfterA)) return;
    }
    persist_phase(p, p.vg[kPassFinish], nullptr,
                  [&](const KArgs<T>& a, int vb, int vg) { body_finish<T, LPR, true>(a, vb, vg); });
    if (!persist_sync(p, kSyncEnd)) return;
    if (!vld(&pc->active)) return;
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

template <typename T, int LPR, int W>
bool fill_kernels(KernelSet* ks) {
  ks->start = (void*)k_start<T, LPR, W>;
  ks->cg_a = (void*)k_cg_a<T, LPR, W>;
  ks->cg_b = (void*)k_cg_b<T, LPR>;
  ks->finish = (void*)k_finish<T, LPR>;
  ks->energy = (void*)k_energy<T, LPR>;
  ks->energy_check = (void*)k_energy_check<T, LPR>;
  ks->init_rng = (void*)k_init_rng<T>;
  ks->scatter_in = (void*)k_scatter_in<T>;
  ks->gather_out = (void*)k_gather_out<T>;
  ks->labels = (void*)k_labels<T>;
  ks->b_start = (void*)kb_start<T, LPR, W>;
  ks->b_cg_a = (void*)kb_cg_a<T, LPR, W>;
  ks->b_cg_b = (void*)kb_cg_b<T, LPR>;
  ks->b_finish = (void*)kb_finish<T, LPR>;
  ks->b_energy_check = (void*)kb_energy_check<T, LPR>;
  ks->b_vote = (void*)k_batch_vote<T>;
  ks->persist = (void*)k_persist<T, LPR, W>;
  ks->smem_start = row_stage_smem<StartStage<T, LPR, W>>();
  {
    const unsigned f0 = row_stage_smem<CgAStage<T, LPR, W, kCgFirst>>();
    const unsigned f1 = row_stage_smem<CgAStage<T, LPR, W, kCgEven>>();
    const unsigned f2 = row_stage_smem<CgAStage<T, LPR, W, kCgOdd>>();
    ks->smem_cg_a = f0 > f1 ? (f0 > f2 ? f0 : f2) : (f1 > f2 ? f1 : f2);
  }
  return true;
}

template <typename T, int LPR>
bool fill_kernels_w(int w, KernelSet* ks) {
  if (w == 8) return fill_kernels<T, LPR, 8>(ks);
  if (w == 16) return fill_kernels<T, LPR, 16>(ks);
  return false;
}

}  // namespace segimpl
