// seg_s_eps_noalloc: the S_eps / coupling-integral evaluation of the energy
// pass for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// is reserved up front by another framework's pool, code that runs while a
// CUDA graph is being captured (allocation is not allowed during capture), or
// a loop with a latency budget that an allocation could break.  This entry
// point takes only caller-owned inputs and outputs; the scratch it needs (one
// partial sum per block and component, plus a completion ticket) lives in a
// file-scope device array of fixed size that every GPU loading the library
// keeps until the process exits.  The paper has no counterpart of this call.
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace segimpl {

namespace {

constexpr int kNaBlocks = 256;                         // grid size (fixed)
constexpr int kNaMaxCols = kMaxCols;                   // components supported
constexpr int kNaTicket = kNaBlocks * kNaMaxCols;      // offset of the ticket
constexpr int kNaScratchDoubles = kNaTicket + 32;      // 8 224 doubles = 64.25 KiB

// Scratch shared by every call on a device: [kNaMaxCols][kNaBlocks] partial
// sums, then the ticket counter.  Host code must not take its address
// directly (the host-side name is only a stand-in): the device address comes
// from cudaGetSymbolAddress.
static __device__ __align__(256) double g_seg_noalloc_scratch[kNaScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Per triangle and component i: int_T u_i^2 sum_{j != i} u_j^2 from the
// barycentric moments (the formula of the energy pass), u in the caller's
// layout u[z * m + i] (float64, not padded, not permuted), |T| from xyz.
template <int LPR>
__global__ void __launch_bounds__(kBlockThreads) k_s_eps_noalloc(const double* __restrict__ u, int nv, int m,
                                                                  const double* __restrict__ xyz,
                                                                  const int* __restrict__ tri, int ntri,
                                                                  double inv_eps2, double* scratch,
                                                                  double* out) {
  constexpr int VW = 2;
  constexpr int NW = kBlockThreads / 32;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rs = lane / LPR, cg = lane % LPR, c0 = cg * VW, lbase = lane - cg;
  const int per_block = (ntri + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per_block;
  const int t1 = min(ntri, t0 + per_block);
  double acc[VW] = {0.0, 0.0};
  for (int base = t0 + warp * RPW; base < t1; base += NW * RPW) {
    const int t = base + rs;
    const bool valid = t < t1;
    double a[3][VW];
    double area = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int v = 0; v < VW; ++v) a[k][v] = 0.0;
    int z[3] = {0, 0, 0};
    bool inside = valid;
    if (valid) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        z[k] = tri[3 * (size_t)t + k];
        inside = inside && z[k] >= 0 && z[k] < nv;
      }
    }
    if (inside) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int v = 0; v < VW; ++v)
          if (c0 + v < m) a[k][v] = u[(size_t)z[k] * m + c0 + v];
      }
      double e1[3], e2[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        e1[d] = xyz[3 * (size_t)z[1] + d] - xyz[3 * (size_t)z[0] + d];
        e2[d] = xyz[3 * (size_t)z[2] + d] - xyz[3 * (size_t)z[0] + d];
      }
      const double cx = e1[1] * e2[2] - e1[2] * e2[1];
      const double cy = e1[2] * e2[0] - e1[0] * e2[2];
      const double cz = e1[0] * e2[1] - e1[1] * e2[0];
      area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    }
    double P[6][VW], E[6][VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      P[0][v] = a[0][v] * a[0][v];
      P[1][v] = a[1][v] * a[1][v];
      P[2][v] = a[2][v] * a[2][v];
      P[3][v] = a[0][v] * a[1][v];
      P[4][v] = a[0][v] * a[2][v];
      P[5][v] = a[1][v] * a[2][v];
    }
    row_exclusive<double, LPR, 6>(P, E, lbase, cg);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const double a0 = a[0][v], a1 = a[1][v], a2 = a[2][v];
      const double e00 = E[0][v], e11 = E[1][v], e22 = E[2][v], e01 = E[3][v], e02 = E[4][v], e12 = E[5][v];
      const double s = a0 + a1 + a2;
      const double q0 = a0 * a0, q1 = a1 * a1, q2 = a2 * a2;
      const double aa = q0 + q1 + q2;
      const double b1x = e00 + e01 + e02, b1y = e01 + e11 + e12, b1z = e02 + e12 + e22;
      const double SB = b1x + b1y + b1z, trB = e00 + e11 + e22;
      const double aB1 = a0 * b1x + a1 * b1y + a2 * b1z;
      const double aBa = q0 * e00 + q1 * e11 + q2 * e22 + 2.0 * (a0 * a1 * e01 + a0 * a2 * e02 + a1 * a2 * e12);
      const double a2B1 = q0 * b1x + q1 * b1y + q2 * b1z;
      const double dBa = a0 * e00 + a1 * e11 + a2 * e22;
      const double a2dB = q0 * e00 + q1 * e11 + q2 * e22;
      const double F = (s * s + aa) * (SB + trB) + 4.0 * s * aB1 + 2.0 * aBa + 4.0 * a2B1 + 4.0 * s * dBa +
                       6.0 * a2dB;
      acc[v] += area * (1.0 / 360.0) * F;
    }
  }
  // warp, then block reduction per component (fixed order)
#pragma unroll
  for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
    for (int v = 0; v < VW; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
  __shared__ double red[NW][kNaMaxCols];
  __shared__ unsigned int ticket;
  if (lane < LPR) {
#pragma unroll
    for (int v = 0; v < VW; ++v) red[warp][c0 + v] = acc[v];
  }
  __syncthreads();
  const int G = gridDim.x;
  const int ms = LPR * VW;
  for (int c = threadIdx.x; c < ms; c += kBlockThreads) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += red[w][c];
    scratch[(size_t)c * G + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaTicket);
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != (unsigned int)(G - 1)) return;
  __threadfence();
  __shared__ double tot[kNaMaxCols];
  for (int c = warp; c < ms; c += NW) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += __ldcg(&scratch[(size_t)c * G + b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) tot[c] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    for (int c = 0; c < m; ++c) {
      out[1 + c] = tot[c];
      S += tot[c];
    }
    out[0] = S * inv_eps2;
    *counter = 0u;
  }
}

}  // namespace

}  // namespace segimpl

using namespace segimpl;

extern "C" seg_status seg_s_eps_noalloc(const double* u, int64_t n_vert, int32_t m, const double* xyz,
                                        const int32_t* tri, int64_t n_tri, double eps, double* out,
                                        void* cuda_stream) {
  auto fail = [](seg_status code, const char* msg) {
    set_last_error(msg);
    return code;
  };
  if (!u || !xyz || !tri || !out) return fail(SEG_ERR_ARG, "seg_s_eps_noalloc: a pointer argument is NULL");
  if (m < 1) return fail(SEG_ERR_ARG, "seg_s_eps_noalloc: m must be >= 1");
  if (m > kNaMaxCols)
    return fail(SEG_ERR_UNSUPPORTED,
                "seg_s_eps_noalloc: m exceeds the 32 components its static scratch array holds");
  if (n_vert < 3 || n_tri < 1 || n_vert > 0x7fffffff || n_tri > 0x7fffffff)
    return fail(SEG_ERR_ARG, "seg_s_eps_noalloc: n_vert must be in [3, 2^31) and n_tri in [1, 2^31)");
  if (!(eps > 0)) return fail(SEG_ERR_ARG, "seg_s_eps_noalloc: eps must be positive");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SEG_ERR_UNSUPPORTED, "seg_s_eps_noalloc: device index too large");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      // once per device, with that device current: resolve the device address
      e = cudaGetSymbolAddress((void**)&g_scratch_addr[dev], g_seg_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return fail(SEG_ERR_CUDA, cudaGetErrorString(e));
      }
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // the ticket counter must start at zero (earlier calls leave it at zero,
  // but an interrupted call could not have reset it)
  e = cudaMemsetAsync(scratch + kNaTicket, 0, sizeof(unsigned int), stream);
  if (e != cudaSuccess) return fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  int lpr = (m + 1) / 2;
  int pw = 1;
  while (pw < lpr) pw <<= 1;
  const double inv_eps2 = 1.0 / (eps * eps);
  const int n = (int)n_tri;
  const int nv = (int)n_vert;
  void* fn = pw == 1   ? (void*)k_s_eps_noalloc<1>
             : pw == 2 ? (void*)k_s_eps_noalloc<2>
             : pw == 4 ? (void*)k_s_eps_noalloc<4>
             : pw == 8 ? (void*)k_s_eps_noalloc<8>
                       : (void*)k_s_eps_noalloc<16>;
  void* args[] = {(void*)&u, (void*)&nv, (void*)&m, (void*)&xyz, (void*)&tri, (void*)&n, (void*)&inv_eps2,
                  (void*)&scratch, (void*)&out};
  // the launch's own status: an error left pending on this thread by earlier,
  // unrelated work is neither reported as ours nor cleared
  e = cudaLaunchKernel(fn, dim3(kNaBlocks), dim3(kBlockThreads), args, 0, stream);
  if (e != cudaSuccess) return fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  return SEG_OK;
}
