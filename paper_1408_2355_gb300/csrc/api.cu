// C ABI of the library (declared in include/seg.h): handles, validation,
// device buffers, the CUDA graph of one step of Algorithm 2.2, batches and the
// launch-geometry autotuner.
//
// The step graph is
//     k_start -> k_energy_check -> k_cg_a -> (k_cg_b -> k_cg_a) x (cg_peel - 1)
//             -> WHILE(cond) { (k_cg_b -> k_cg_a) x kCgUnroll } -> k_finish
// where the WHILE node's condition (CG pass B needed next) is set on the
// device by the last block of k_start (any component still above tolerance),
// k_energy_check (stop rule), the first k_cg_a of a solve (its only iteration
// converged) and k_cg_b (convergence / iteration cap); passes after the loop
// has ended return at once.  A step whose solve ends in its first pass A runs
// no pass B at all.  A whole step -- including the data-dependent CG
// iteration count -- runs without a host round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "seg_internal.h"

using namespace segimpl;

namespace {

thread_local std::string g_err;

seg_status fail(seg_status code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define SEG_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(SEG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

void segimpl::set_last_error(const char* msg) { g_err = msg; }
const char* segimpl::last_error() { return g_err.c_str(); }

struct seg_mesh {
  HostMesh h;
};

struct seg_problem {
  int64_t n = 0, nnz = 0, f = 0;
  double tau = 0, area = 0;
  seg_precision prec = SEG_FP64;
  int device = 0;
  int ell_w = 8;
  uint32_t flags = 0;  // seg_assemble_ex flags
  int* ell_col = nullptr;
  void* valA = nullptr;
  void* valM = nullptr;
  void* valK = nullptr;
  void* dinv = nullptr;
  void* diagA = nullptr;
  int* tri = nullptr;
  void* tarea = nullptr;
  int* perm = nullptr;
  int* iperm = nullptr;
};

struct seg_state {
  const seg_problem* p = nullptr;
  int m = 0, ms = 0, lpr = 0;
  double eps = 0;
  seg_precision prec = SEG_FP64;
  double cg_rtol = 0;
  int cg_maxit = 0;
  long long check_every = 0;
  double energy_tol = 0;
  double energy_rtol = 0;
  long long max_steps = 0;
  unsigned long long wait_ns = kDefaultWaitNs;  // limit of one bounded device wait
  int stall_waits = 0;                          // seg_set_wait_stall
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int launch_mode = 0;
  int grid[4] = {0, 0, 0, 0};  // blocks of the row kernels: start, CG pass A, CG pass B, finish
  int grid_e = 0;   // blocks of the S_eps check kernel
  int grid_cap = 0;    // the partial-sum buffer holds this many row blocks
  int grid_e_cap = 0;  // ... and this many triangle blocks
  void* X = nullptr;
  void* Y = nullptr;        // correction of the CG iterate (x = X + y), starts at a prediction
  void* H0 = nullptr;       // the last two (float) or three (double) steps' final corrections
  void* H1 = nullptr;
  void* H2 = nullptr;       // double states only
  void* Z = nullptr;        // preconditioned residual
  void* P0 = nullptr;       // search directions, ping-pong
  void* P1 = nullptr;
  void* Q = nullptr;
  DevCtl* ctl = nullptr;
  void* part = nullptr;
  double* io = nullptr;     // n * m float64 staging
  double* ones = nullptr;   // kMaxCols ones (scale reset)
  double* scale_backup = nullptr;
  int* am = nullptr;
  unsigned char* vp = nullptr;
  DevCtl* hctl = nullptr;   // pinned mirror
  KernelSet ks{};
  KArgs<float> af{};
  KArgs<double> ad{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  bool pending = true;      // inv_n must be recomputed before use
  int cg_peel = kCgPeelDefault;  // CG iterations of the step graph before its WHILE node
  long long peel_step = 0;       // step and CG iteration counters when the peel was last reviewed
  long long peel_it = 0;
  // step graphs replaced while launches of them may still be in flight
  // (destroyed once the stream has drained)
  std::vector<std::pair<cudaGraph_t, cudaGraphExec_t>> retired;
  long long* hsnap = nullptr;   // pinned: counters after a chunk of seg_step, 2 slots x (step, cg_total)
  cudaEvent_t snap_ev[2] = {nullptr, nullptr};
  DevCtl* hring = nullptr;      // pinned: SEG_STATS_RING control-block copies of seg_stats_enqueue
  cudaEvent_t ring_ev[SEG_STATS_RING] = {};
  int ring_ticket[SEG_STATS_RING] = {};  // ticket whose copy a slot holds (-1: none)
  int ring_next = 0;
};

namespace {

size_t vsize(seg_precision p) { return p == SEG_MIXED_FP32 ? sizeof(float) : sizeof(double); }

// P1 interpolation onto a refined mesh (caller numbering, float64):
// uf[z][i] = (uc[a][i] + uc[b][i]) / 2 with (a, b) = parents of z.
__global__ void k_prolong(const double* uc, const int32_t* parents, double* uf, long long nf, int m) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf * m) return;
  const long long z = k / m;
  const int i = (int)(k % m);
  const long long a = parents[2 * z], b = parents[2 * z + 1];
  uf[k] = 0.5 * (uc[a * m + i] + uc[b * m + i]);
}

// Bytes of the partial-sum buffer: up to kMaxDots * ms sums over `grid` row
// blocks or one sum over `grid_e` triangle blocks (8-byte parts).
size_t partial_bytes(int ms, int grid, int grid_e) {
  return std::max((size_t)kMaxDots * ms * grid, (size_t)grid_e) * 8;
}

template <typename T>
KArgs<T>& args_of(seg_state* s);
template <>
KArgs<float>& args_of<float>(seg_state* s) { return s->af; }
template <>
KArgs<double>& args_of<double>(seg_state* s) { return s->ad; }

struct Launch {
  int set_cond = 0, force = 0, apply_x = 0, apply_ode = 0, count_step = 0, ignore_halt = 1, norm_only = 0;
};

template <typename T>
KArgs<T> make_args(seg_state* s, const Launch& l) {
  KArgs<T> a = args_of<T>(s);
  a.set_cond = l.set_cond;
  a.cond = (unsigned long long)s->cond;
  a.force = l.force;
  a.apply_x = l.apply_x;
  a.apply_ode = l.apply_ode;
  a.count_step = l.count_step;
  a.ignore_halt = l.ignore_halt;
  a.norm_only = l.norm_only;
  return a;
}

// Dynamic shared memory of a row kernel (the TMA-staged ones use some).
unsigned smem_of(const seg_state* s, void* fn) {
  if (fn == s->ks.start) return s->ks.smem_start;
  if (fn == s->ks.cg_a) return s->ks.smem_cg_a;
  return 0;
}

int grid_of(const seg_state* s, void* fn) {
  if (fn == s->ks.energy_check || fn == s->ks.energy) return s->grid_e;
  if (fn == s->ks.start) return s->grid[kPassStart];
  if (fn == s->ks.cg_a) return s->grid[kPassCgA];
  if (fn == s->ks.cg_b) return s->grid[kPassCgB];
  return s->grid[kPassFinish];
}

// Launch one row kernel with the state's arguments.
seg_status launch_row(seg_state* s, void* fn, const Launch& l) {
  cudaError_t e;
  const unsigned smem = smem_of(s, fn);
  const dim3 grid(grid_of(s, fn));
  if (s->prec == SEG_MIXED_FP32) {
    KArgs<float> a = make_args<float>(s, l);
    void* args[] = {&a};
    e = cudaLaunchKernel(fn, grid, dim3(kBlockThreads), args, smem, s->stream);
  } else {
    KArgs<double> a = make_args<double>(s, l);
    void* args[] = {&a};
    e = cudaLaunchKernel(fn, grid, dim3(kBlockThreads), args, smem, s->stream);
  }
  if (e != cudaSuccess) return fail(SEG_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return SEG_OK;
}

// Launch an element-wise auxiliary kernel over `count` items with extra args.
template <typename... Extra>
seg_status launch_aux(seg_state* s, void* fn, long long count, Extra... extra) {
  const int bt = 256;
  const long long blocks = (count + bt - 1) / bt;
  if (blocks == 0) return SEG_OK;
  cudaError_t e;
  if (s->prec == SEG_MIXED_FP32) {
    KArgs<float> a = make_args<float>(s, Launch());
    void* args[] = {&a, &extra...};
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(bt), args, 0, s->stream);
  } else {
    KArgs<double> a = make_args<double>(s, Launch());
    void* args[] = {&a, &extra...};
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(bt), args, 0, s->stream);
  }
  if (e != cudaSuccess) return fail(SEG_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return SEG_OK;
}

seg_status sync_ctl(seg_state* s) {
  SEG_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->stream));
  SEG_CUDA(cudaStreamSynchronize(s->stream));
  return SEG_OK;
}

// Recompute the normalisation factors of the stored state if needed (fused
// Algorithm 2.2 step 3 of the previous step / of freshly set data).  The
// start pass runs in its norm-only form: the solver's state for the next
// step is left as it is, so reading the state does not change the run.
seg_status ensure_norm(seg_state* s) {
  if (!s->pending) return SEG_OK;
  Launch l;
  l.norm_only = 1;
  seg_status st = launch_row(s, s->ks.start, l);
  if (st != SEG_OK) return st;
  s->pending = false;
  return SEG_OK;
}

// One step with the kernels of the step graph launched one by one: the CG
// loop condition is read back by the host after every iteration.
seg_status direct_step(seg_state* s) {
  Launch l;
  l.ignore_halt = 0;
  seg_status st = launch_row(s, s->ks.start, l);
  if (st == SEG_OK) st = launch_row(s, s->ks.energy_check, l);
  if (st == SEG_OK) st = sync_ctl(s);
  while (st == SEG_OK && s->hctl->cont && !s->hctl->halted &&
         !(s->max_steps > 0 && s->hctl->step >= s->max_steps)) {
    st = launch_row(s, s->ks.cg_a, l);
    if (st == SEG_OK) st = launch_row(s, s->ks.cg_b, l);
    if (st == SEG_OK) st = sync_ctl(s);
  }
  Launch f = l;
  f.apply_x = 1;
  f.apply_ode = 1;
  f.count_step = 1;
  if (st == SEG_OK) st = launch_row(s, s->ks.finish, f);
  return st;
}

// Mean duration of `reps` back-to-back launches of hot-path kernel `which`
// (see seg_time_kernel) on the state's buffers, after one warm-up launch.
seg_status time_launches(seg_state* s, int which, int reps, double* ms_per_launch) {
  void* fns[] = {s->ks.start,        s->ks.cg_a,   s->ks.cg_b,   s->ks.finish, s->ks.energy_check,
                 s->ks.energy,       s->ks.cg_a,   s->ks.finish, s->ks.cg_a,   s->ks.cg_b};
  if (which != 0 && which != 4 && which != 5) {
    // the iteration count the pass sees selects its form: CG pass A as the
    // first iteration of a solve (1), an odd one (6: also the two pending
    // solution updates) or a later even one (8); CG pass B in a later
    // iteration (2) or the first (9: also copies p_1 = z_0); the finish pass
    // with one pending update (3) or two (7, after an odd count of 3 or more).
    // Forced launches leave the count as it is.
    static const int it_of[] = {0, 0, 1, 2, 0, 0, 1, 3, 2, 0};
    const int it = it_of[which];
    SEG_CUDA(cudaMemcpyAsync(&s->ctl->it, &it, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    SEG_CUDA(cudaStreamSynchronize(s->stream));
  }
  Launch l;
  l.force = 1;
  l.apply_x = 1;
  l.apply_ode = 1;
  cudaEvent_t e0, e1;
  SEG_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SEG_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
  }
  seg_status st = launch_row(s, fns[which], l);  // warm-up
  if (st == SEG_OK) {
    cudaEventRecord(e0, s->stream);
    for (int r = 0; r < reps && st == SEG_OK; ++r) st = launch_row(s, fns[which], l);
    cudaEventRecord(e1, s->stream);
  }
  ce = cudaEventSynchronize(e1);
  float ms = 0;
  if (st == SEG_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SEG_OK) return st;
  if (ce != cudaSuccess) return fail(SEG_ERR_CUDA, std::string("event timing: ") + cudaGetErrorString(ce));
  *ms_per_launch = ms / reps;
  return SEG_OK;
}

seg_status status_from_ctl(const DevCtl& c) {
  if (c.status & 4) return fail(SEG_ERR_TIMEOUT, "a bounded wait for staged data timed out; the run was halted");
  if (c.status & 2) return fail(SEG_ERR_NONFINITE, "a norm, inner product or energy became non-finite (or a component vanished)");
  if (c.status & 1) return fail(SEG_ERR_NOT_CONVERGED, "a step-1 CG solve reached cg_maxit before cg_rtol");
  return SEG_OK;
}

template <typename T>
cudaError_t add_kernel_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                            void* fn, int grid, const KArgs<T>& a, unsigned smem) {
  KArgs<T> copy = a;
  void* args[] = {&copy};
  cudaKernelNodeParams kp{};
  kp.func = fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(kBlockThreads);
  kp.sharedMemBytes = smem;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

template <typename T>
seg_status build_graph_t(seg_state* s) {
  SEG_CUDA(cudaGraphCreate(&s->graph, 0));
  SEG_CUDA(cudaGraphConditionalHandleCreate(&s->cond, s->graph, 0, cudaGraphCondAssignDefault));
  Launch l;
  l.set_cond = 1;
  l.ignore_halt = 0;
  KArgs<T> base = make_args<T>(s, l);
  cudaGraphNode_t n_start, n_energy, n_loop, n_a, n_b, n_fin;
  SEG_CUDA(add_kernel_node<T>(&n_start, s->graph, nullptr, 0, s->ks.start, s->grid[kPassStart], base,
                              s->ks.smem_start));
  SEG_CUDA(add_kernel_node<T>(&n_energy, s->graph, &n_start, 1, s->ks.energy_check, s->grid_e, base, 0));
  // the first cg_peel CG iterations are plain graph nodes (a pass after the
  // loop has ended returns at once), the rest a WHILE node: an evaluation of
  // the loop condition costs more than a pass that returns at once.  An
  // iteration's pass B comes after the loop's condition, so that a solve
  // that ends in its first pass A launches no pass B.
  SEG_CUDA(add_kernel_node<T>(&n_a, s->graph, &n_energy, 1, s->ks.cg_a, s->grid[kPassCgA], base, s->ks.smem_cg_a));
  cudaGraphNode_t last = n_a;
  for (int u = 1; u < s->cg_peel; ++u) {
    SEG_CUDA(add_kernel_node<T>(&n_b, s->graph, &last, 1, s->ks.cg_b, s->grid[kPassCgB], base, 0));
    SEG_CUDA(add_kernel_node<T>(&n_a, s->graph, &n_b, 1, s->ks.cg_a, s->grid[kPassCgA], base, s->ks.smem_cg_a));
    last = n_a;
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = s->cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  SEG_CUDA(cudaGraphAddNode(&n_loop, s->graph, &last, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  // kCgUnroll CG iterations per evaluation of the loop condition, each the
  // pass B of one iteration and the pass A of the next; passes after the
  // loop has ended return at once (ctl->cont == 0)
  cudaGraphNode_t prev = nullptr;
  for (int u = 0; u < kCgUnroll; ++u) {
    SEG_CUDA(add_kernel_node<T>(&n_b, body, prev ? &prev : nullptr, prev ? 1 : 0, s->ks.cg_b, s->grid[kPassCgB],
                                base, 0));
    SEG_CUDA(add_kernel_node<T>(&n_a, body, &n_b, 1, s->ks.cg_a, s->grid[kPassCgA], base, s->ks.smem_cg_a));
    prev = n_a;
  }
  KArgs<T> fin = base;
  fin.apply_x = 1;
  fin.apply_ode = 1;
  fin.count_step = 1;
  SEG_CUDA(add_kernel_node<T>(&n_fin, s->graph, &n_loop, 1, s->ks.finish, s->grid[kPassFinish], fin, 0));
  SEG_CUDA(cudaGraphInstantiate(&s->exec, s->graph, 0));
  return SEG_OK;
}

template <typename T>
void fill_args(seg_state* s) {
  const seg_problem* p = s->p;
  KArgs<T>& a = args_of<T>(s);
  a = KArgs<T>{};
  a.n = (int)p->n;
  a.m = s->m;
  a.ms = s->ms;
  a.ell_w = p->ell_w;
  a.ell_col = p->ell_col;
  a.valA = (const T*)p->valA;
  a.valM = (const T*)p->valM;
  a.valK = (const T*)p->valK;
  a.dinv = (const T*)p->dinv;
  a.X = (T*)s->X;
  a.Y = (T*)s->Y;
  a.H0 = (T*)s->H0;
  a.H1 = (T*)s->H1;
  a.H2 = (T*)s->H2;
  a.diagA = (const T*)p->diagA;
  a.Z = (T*)s->Z;
  a.P0 = (T*)s->P0;
  a.P1 = (T*)s->P1;
  a.Q = (T*)s->Q;
  a.ctl = s->ctl;
  a.part = s->part;
  a.tau = p->tau;
  a.coef = 2.0 * p->tau / (s->eps * s->eps);
  a.inv_eps2 = 1.0 / (s->eps * s->eps);
  a.rtol2 = s->cg_rtol * s->cg_rtol;
  a.maxit = s->cg_maxit;
  a.tri = p->tri;
  a.tarea = (const T*)p->tarea;
  a.ntri = (int)p->f;
  a.check_every = s->check_every;
  a.energy_tol = s->energy_tol;
  a.energy_rtol = s->energy_rtol;
  a.max_steps = s->max_steps;
  a.wait_ns = s->wait_ns;
  a.stall_waits = s->stall_waits;
}

template <typename T>
seg_status upload_vals(const std::vector<double>& src, void** dst) {
  std::vector<T> tmp(src.begin(), src.end());
  SEG_CUDA(cudaMalloc(dst, tmp.size() * sizeof(T)));
  SEG_CUDA(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SEG_OK;
}

seg_status upload_vals_prec(seg_precision prec, const std::vector<double>& src, void** dst) {
  return prec == SEG_MIXED_FP32 ? upload_vals<float>(src, dst) : upload_vals<double>(src, dst);
}

template <typename I>
seg_status upload_ints(const std::vector<I>& src, I** dst) {
  SEG_CUDA(cudaMalloc((void**)dst, std::max<size_t>(1, src.size()) * sizeof(I)));
  if (!src.empty()) SEG_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(I), cudaMemcpyHostToDevice));
  return SEG_OK;
}

void drop_retired(seg_state* s) {
  for (auto& r : s->retired) {
    if (r.second) cudaGraphExecDestroy(r.second);
    if (r.first) cudaGraphDestroy(r.first);
  }
  s->retired.clear();
}

void drop_graph(seg_state* s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->exec = nullptr;
  s->graph = nullptr;
}

// Set the graph aside (launches of it may be in flight); the next graph-mode
// step builds a new one.
void retire_graph(seg_state* s) {
  if (s->exec || s->graph) s->retired.emplace_back(s->graph, s->exec);
  s->exec = nullptr;
  s->graph = nullptr;
}

void free_state(seg_state* s) {
  if (!s) return;
  drop_retired(s);
  drop_graph(s);
  void* bufs[] = {s->X, s->Y, s->H0, s->H1, s->H2, s->Z, s->P0, s->P1, s->Q, s->ctl, s->part, s->io, s->ones, s->scale_backup, s->am, s->vp};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (s->hctl) cudaFreeHost(s->hctl);
  if (s->hsnap) cudaFreeHost(s->hsnap);
  for (cudaEvent_t e : s->snap_ev)
    if (e) cudaEventDestroy(e);
  if (s->hring) cudaFreeHost(s->hring);
  for (cudaEvent_t e : s->ring_ev)
    if (e) cudaEventDestroy(e);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

seg_status reset_ctl(seg_state* s) {
  SEG_CUDA(cudaMemsetAsync(s->ctl, 0, sizeof(DevCtl), s->stream));
  s->pending = true;
  return SEG_OK;
}

}  // namespace

extern "C" {

const char* seg_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ meshes

seg_status seg_create_mesh(const double* xyz, int64_t n_vert, const int32_t* tri, int64_t n_tri,
                           seg_mesh** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!xyz || !tri) return fail(SEG_ERR_ARG, "xyz or tri is NULL");
  if (n_vert < 3 || n_tri < 1 || n_vert > (int64_t)1 << 30 || n_tri > (int64_t)1 << 30)
    return fail(SEG_ERR_ARG, "mesh sizes out of range");
  seg_mesh* m = new (std::nothrow) seg_mesh;
  if (!m) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  m->h.n = n_vert;
  m->h.f = n_tri;
  m->h.xyz.assign(xyz, xyz + 3 * n_vert);
  m->h.tri.assign(tri, tri + 3 * n_tri);
  seg_status code;
  std::string msg = validate_mesh(m->h, &code);
  if (code != SEG_OK) {
    delete m;
    return fail(code, msg);
  }
  *out = m;
  return SEG_OK;
}

seg_status seg_mesh_icosphere(int32_t level, seg_mesh** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (level < 0 || level > 10) return fail(SEG_ERR_ARG, "icosphere level must be in [0, 10]");
  seg_mesh* m = new (std::nothrow) seg_mesh;
  if (!m) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  make_icosphere(level, &m->h);
  *out = m;
  return SEG_OK;
}

seg_status seg_mesh_ellipsoid(int32_t level, double a, double b, double c, seg_mesh** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!(a > 0 && b > 0 && c > 0)) return fail(SEG_ERR_ARG, "semi-axes must be positive");
  seg_status st = seg_mesh_icosphere(level, out);
  if (st != SEG_OK) return st;
  std::vector<double>& x = (*out)->h.xyz;
  for (int64_t v = 0; v < (*out)->h.n; ++v) {
    double* p = &x[3 * v];
    double q = std::sqrt((p[0] / a) * (p[0] / a) + (p[1] / b) * (p[1] / b) + (p[2] / c) * (p[2] / c));
    p[0] /= q;
    p[1] /= q;
    p[2] /= q;
  }
  return SEG_OK;
}

seg_status seg_mesh_torus(int32_t nu, int32_t nv, double R, double r, seg_mesh** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nu < 3 || nv < 3 || (int64_t)nu * nv > (int64_t)1 << 29) return fail(SEG_ERR_ARG, "torus grid out of range");
  if (!(r > 0 && R > r)) return fail(SEG_ERR_ARG, "torus radii need R > r > 0");
  seg_mesh* m = new (std::nothrow) seg_mesh;
  if (!m) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  make_torus(nu, nv, R, r, &m->h);
  *out = m;
  return SEG_OK;
}

seg_status seg_mesh_dziuk(int32_t level, seg_mesh** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (level < 0 || level > 10) return fail(SEG_ERR_ARG, "surface (D) level must be in [0, 10]");
  seg_mesh* m = new (std::nothrow) seg_mesh;
  if (!m) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  make_dziuk(level, &m->h);
  *out = m;
  return SEG_OK;
}

seg_status seg_mesh_refine(const seg_mesh* coarse, const seg_surface* surf, seg_mesh** fine, int32_t* parents) {
  if (!fine) return fail(SEG_ERR_ARG, "fine is NULL");
  *fine = nullptr;
  if (!coarse || !surf) return fail(SEG_ERR_ARG, "coarse mesh or surface is NULL");
  if (surf->reserved != 0) return fail(SEG_ERR_ARG, "surface.reserved must be 0");
  if (surf->kind < SEG_SURFACE_NONE || surf->kind > SEG_SURFACE_DZIUK) return fail(SEG_ERR_ARG, "unknown surface kind");
  if (surf->kind == SEG_SURFACE_ELLIPSOID && !(surf->p0 > 0 && surf->p1 > 0 && surf->p2 > 0))
    return fail(SEG_ERR_ARG, "ellipsoid semi-axes must be positive");
  if (surf->kind == SEG_SURFACE_TORUS && !(surf->p1 > 0 && surf->p0 > surf->p1))
    return fail(SEG_ERR_ARG, "torus radii need p0 > p1 > 0");
  const HostMesh& h = coarse->h;
  // fine sizes: n + edges <= n + 3f, 4f triangles; keep 32-bit indices
  if (h.n + 3 * h.f >= ((int64_t)1 << 31) || 4 * h.f >= ((int64_t)1 << 31))
    return fail(SEG_ERR_ARG, "refined mesh would exceed 32-bit indices");
  seg_mesh* m = new (std::nothrow) seg_mesh;
  if (!m) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  std::vector<int32_t> par;
  refine_mesh(h, SurfaceDesc{surf->kind, surf->p0, surf->p1, surf->p2}, &m->h, parents ? &par : nullptr);
  if (parents) std::copy(par.begin(), par.end(), parents);
  *fine = m;
  return SEG_OK;
}

seg_status seg_mesh_info(const seg_mesh* mesh, int64_t* n_vert, int64_t* n_tri) {
  if (!mesh) return fail(SEG_ERR_ARG, "mesh is NULL");
  if (n_vert) *n_vert = mesh->h.n;
  if (n_tri) *n_tri = mesh->h.f;
  return SEG_OK;
}

seg_status seg_mesh_get(const seg_mesh* mesh, double* xyz, int32_t* tri) {
  if (!mesh) return fail(SEG_ERR_ARG, "mesh is NULL");
  if (xyz) std::memcpy(xyz, mesh->h.xyz.data(), mesh->h.xyz.size() * sizeof(double));
  if (tri) std::memcpy(tri, mesh->h.tri.data(), mesh->h.tri.size() * sizeof(int32_t));
  return SEG_OK;
}

void seg_mesh_destroy(seg_mesh* mesh) { delete mesh; }

// ---------------------------------------------------------------- assembly

seg_status seg_assemble(const seg_mesh* mesh, double tau, seg_precision precision, seg_problem** out) {
  return seg_assemble_ex(mesh, tau, precision, 0u, out);
}

seg_status seg_assemble_ex(const seg_mesh* mesh, double tau, seg_precision precision, uint32_t flags,
                           seg_problem** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh) return fail(SEG_ERR_ARG, "mesh is NULL");
  if (!(tau > 0) || !std::isfinite(tau)) return fail(SEG_ERR_ARG, "tau must be positive and finite");
  if (precision != SEG_FP64 && precision != SEG_MIXED_FP32) return fail(SEG_ERR_ARG, "unknown precision");
  if (flags & ~(uint32_t)SEG_ASSEMBLE_LUMPED_MASS) return fail(SEG_ERR_ARG, "unknown assembly flag");
  HostCSR csr;
  assemble_p1(mesh->h, &csr);
  const int64_t n = csr.n;
  if (flags & SEG_ASSEMBLE_LUMPED_MASS) {
    // M_L = diag(row sums of M); the sparsity pattern stays (K uses it)
    for (int64_t i = 0; i < n; ++i) {
      double rs = 0.0;
      for (int32_t e = csr.rowptr[i]; e < csr.rowptr[i + 1]; ++e) rs += csr.M[e];
      for (int32_t e = csr.rowptr[i]; e < csr.rowptr[i + 1]; ++e) csr.M[e] = csr.col[e] == i ? rs : 0.0;
    }
  }
  std::vector<double> A(csr.nnz), dinv(n), diag(n);
  for (int64_t e = 0; e < csr.nnz; ++e) A[e] = csr.M[e] + tau * csr.K[e];
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t e = csr.rowptr[i]; e < csr.rowptr[i + 1]; ++e)
      if (csr.col[e] == i) d = A[e];
    if (!(d > 0)) return fail(SEG_ERR_MESH, "non-positive diagonal of M + tau K");
    diag[i] = d;
    dinv[i] = 1.0 / d;
  }
  // padded ELL rows: every row holds W entries (W = 8, or 16 for vertex
  // degrees up to 15); unused entries repeat the row itself with value 0, so
  // kernels read them without a branch (the data there is always finite)
  int32_t max_row = 0;
  for (int64_t i = 0; i < n; ++i) max_row = std::max(max_row, csr.rowptr[i + 1] - csr.rowptr[i]);
  if (max_row > 16) return fail(SEG_ERR_UNSUPPORTED, "a vertex has more than 15 neighbours (padded rows hold 16)");
  const int W = max_row <= 8 ? 8 : 16;
  std::vector<int32_t> ecol((size_t)n * W);
  std::vector<double> eA((size_t)n * W, 0.0), eM((size_t)n * W, 0.0), eK((size_t)n * W, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < W; ++k) ecol[i * W + k] = (int32_t)i;
  for (int64_t i = 0; i < n; ++i) {
    for (int32_t e = csr.rowptr[i], k = 0; e < csr.rowptr[i + 1]; ++e, ++k) {
      ecol[i * W + k] = csr.col[e];
      eA[i * W + k] = A[e];
      eM[i * W + k] = csr.M[e];
      eK[i * W + k] = csr.K[e];
    }
  }
  seg_problem* p = new (std::nothrow) seg_problem;
  if (!p) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  p->ell_w = W;
  p->flags = flags;
  p->n = n;
  p->nnz = csr.nnz;
  p->f = mesh->h.f;
  p->tau = tau;
  p->prec = precision;
  double area = 0;
  for (double a : csr.area) area += a;
  p->area = area;
  cudaError_t e = cudaGetDevice(&p->device);
  seg_status st = SEG_OK;
  if (e != cudaSuccess) st = fail(SEG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (st == SEG_OK) st = upload_ints(ecol, &p->ell_col);
  if (st == SEG_OK) st = upload_vals_prec(precision, eA, &p->valA);
  if (st == SEG_OK) st = upload_vals_prec(precision, eM, &p->valM);
  if (st == SEG_OK) st = upload_vals_prec(precision, eK, &p->valK);
  if (st == SEG_OK) st = upload_vals_prec(precision, dinv, &p->dinv);
  if (st == SEG_OK) st = upload_vals_prec(precision, diag, &p->diagA);
  if (st == SEG_OK) st = upload_ints(csr.tri_rows, &p->tri);
  if (st == SEG_OK) st = upload_vals_prec(precision, csr.area, &p->tarea);
  if (st == SEG_OK) st = upload_ints(csr.perm, &p->perm);
  if (st == SEG_OK) st = upload_ints(csr.iperm, &p->iperm);
  if (st != SEG_OK) {
    seg_problem_destroy(p);
    return st;
  }
  *out = p;
  return SEG_OK;
}

seg_status seg_problem_info(const seg_problem* p, int64_t* n_vert, int64_t* nnz, double* tau, double* area) {
  if (!p) return fail(SEG_ERR_ARG, "problem is NULL");
  if (n_vert) *n_vert = p->n;
  if (nnz) *nnz = p->nnz;
  if (tau) *tau = p->tau;
  if (area) *area = p->area;
  return SEG_OK;
}

void seg_problem_destroy(seg_problem* p) {
  if (!p) return;
  void* bufs[] = {p->ell_col, p->valA, p->valM, p->valK, p->dinv, p->diagA, p->tri, p->tarea, p->perm, p->iperm};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
}

// ------------------------------------------------------------------- state

seg_status seg_state_create(const seg_problem* p, int32_t m, double eps, seg_init init, uint64_t seed,
                            const seg_params* opt, void* cuda_stream, seg_state** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!p) return fail(SEG_ERR_ARG, "problem is NULL");
  if (m < 1) return fail(SEG_ERR_ARG, "m must be >= 1");
  if (m > kMaxCols) return fail(SEG_ERR_UNSUPPORTED, "m must be <= 32");
  if (!(eps > 0) || !std::isfinite(eps)) return fail(SEG_ERR_ARG, "eps must be positive and finite");
  if (init != SEG_INIT_ONEHOT && init != SEG_INIT_UNIFORM) return fail(SEG_ERR_ARG, "unknown init kind");
  SEG_CUDA(cudaSetDevice(p->device));
  seg_state* s = new (std::nothrow) seg_state;
  if (!s) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  s->p = p;
  s->m = m;
  s->eps = eps;
  s->prec = p->prec;
  const int vw = s->prec == SEG_MIXED_FP32 ? 4 : 2;
  int lpr = (m + vw - 1) / vw;
  int pw = 1;
  while (pw < lpr) pw <<= 1;
  s->lpr = pw;
  s->ms = pw * vw;
  if ((int64_t)p->n * 2 * s->ms >= ((int64_t)1 << 31)) {
    delete s;
    return fail(SEG_ERR_UNSUPPORTED, "n_vert * padded m too large for 32-bit row offsets");
  }
  seg_params prm{};
  if (opt) prm = *opt;
  s->cg_rtol = prm.cg_rtol > 0 ? prm.cg_rtol : (s->prec == SEG_MIXED_FP32 ? 1e-7 : 1e-12);
  s->cg_maxit = prm.cg_maxit > 0 ? prm.cg_maxit : 1000;
  s->check_every = prm.check_every > 0 ? prm.check_every
                                       : (prm.check_every < 0 ? 0 : std::max<long long>(1, std::llround(0.1 / p->tau)));
  s->energy_tol = prm.energy_tol > 0 ? prm.energy_tol : (prm.energy_tol < 0 ? -1.0 : 1e-6);
  if (!(prm.energy_rtol >= 0.0) || !std::isfinite(prm.energy_rtol)) {
    delete s;
    return fail(SEG_ERR_ARG, "energy_rtol must be finite and >= 0");
  }
  s->energy_rtol = prm.energy_rtol;
  s->max_steps = prm.max_steps > 0 ? prm.max_steps : 0;
  s->wait_ns = prm.wait_limit_ns > 0 ? (unsigned long long)prm.wait_limit_ns : kDefaultWaitNs;
  if (prm.launch_mode != 0 && prm.launch_mode != 1) {
    delete s;
    return fail(SEG_ERR_ARG, "launch_mode must be 0 (graph) or 1 (direct)");
  }
  if (prm.grid_blocks > kMaxGrid) {
    delete s;
    return fail(SEG_ERR_ARG, "grid_blocks must be at most 2048");
  }
  if (prm.reserved != 0) {
    delete s;
    return fail(SEG_ERR_ARG, "seg_params.reserved must be 0");
  }
  s->launch_mode = prm.launch_mode;
  bool ok = s->prec == SEG_MIXED_FP32 ? get_kernels_f32(s->lpr, p->ell_w, &s->ks)
                                      : get_kernels_f64(s->lpr, p->ell_w, &s->ks);
  if (!ok) {
    delete s;
    return fail(SEG_ERR_UNSUPPORTED, "no kernel specialisation for this m and precision");
  }
  {
    // the TMA-staged kernels may need more than the default 48 KiB
    const void* fns[4] = {s->ks.start, s->ks.cg_a, s->ks.b_start, s->ks.b_cg_a};
    const unsigned sm[4] = {s->ks.smem_start, s->ks.smem_cg_a, s->ks.smem_start, s->ks.smem_cg_a};
    for (int k = 0; k < 4; ++k) {
      cudaError_t fe = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[k]);
      if (fe != cudaSuccess) {
        delete s;
        return fail(SEG_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(fe));
      }
    }
  }
  int nsm = 0;
  cudaError_t ce = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  if (ce != cudaSuccess) {
    delete s;
    return fail(SEG_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(ce));
  }
  // blocks of at least 256 rows (1024 triangles), at most kRowBlocksPerSM
  // (kTriBlocksPerSM) per SM; the geometry is part of the state, so results
  // do not depend on whether the state runs alone or in a batch
  const int g0 = prm.grid_blocks > 0
                     ? prm.grid_blocks
                     : (int)std::min<int64_t>(kRowBlocksPerSM * nsm, std::max<int64_t>(1, (p->n + 255) / 256));
  for (int k = 0; k < 4; ++k) s->grid[k] = g0;
  s->grid_e = (int)std::min<int64_t>(kTriBlocksPerSM * nsm, std::max<int64_t>(1, (p->f + 1023) / 1024));
  s->grid_cap = std::max(g0, std::min(kMaxGrid, kTuneWaves * kRowBlocksPerSM * nsm));
  s->grid_e_cap = std::max(s->grid_e, std::min(kMaxGrid, kTuneWaves * kTriBlocksPerSM * nsm));
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    ce = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      delete s;
      return fail(SEG_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(ce));
    }
    s->own_stream = true;
  }
  const size_t vbytes = (size_t)p->n * s->ms * vsize(s->prec);
  const size_t pbytes = partial_bytes(s->ms, s->grid_cap, s->grid_e_cap);
  struct {
    void** ptr;
    size_t bytes;
  } allocs[] = {{&s->X, vbytes},
                {&s->Y, vbytes},
                {&s->H0, vbytes},
                {&s->H1, vbytes},
                {&s->H2, s->prec == SEG_FP64 ? vbytes : 0},
                {&s->Z, vbytes},
                {&s->P0, vbytes},
                {&s->P1, vbytes},
                {&s->Q, vbytes},
                {(void**)&s->ctl, sizeof(DevCtl)},
                {&s->part, pbytes},
                {(void**)&s->io, std::max<size_t>(8, (size_t)p->n * m * sizeof(double))},
                {(void**)&s->ones, kMaxCols * sizeof(double)},
                {(void**)&s->scale_backup, kMaxCols * sizeof(double)},
                {(void**)&s->am, std::max<size_t>(4, (size_t)p->n * sizeof(int))},
                {(void**)&s->vp, std::max<size_t>(4, (size_t)p->n)}};
  for (auto& al : allocs) {
    if (al.bytes == 0) continue;  // (a buffer only some precisions use)
    ce = cudaMalloc(al.ptr, al.bytes);
    if (ce != cudaSuccess) {
      free_state(s);
      return fail(ce == cudaErrorMemoryAllocation ? SEG_ERR_NO_MEMORY : SEG_ERR_CUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(ce));
    }
    ce = cudaMemsetAsync(*al.ptr, 0, al.bytes, s->stream);
    if (ce != cudaSuccess) {
      free_state(s);
      return fail(SEG_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(ce));
    }
  }
  ce = cudaMallocHost((void**)&s->hctl, sizeof(DevCtl));
  if (ce == cudaSuccess) ce = cudaMallocHost((void**)&s->hsnap, 4 * sizeof(long long));
  if (ce == cudaSuccess) ce = cudaMallocHost((void**)&s->hring, SEG_STATS_RING * sizeof(DevCtl));
  if (ce != cudaSuccess) {
    free_state(s);
    return fail(SEG_ERR_NO_MEMORY, std::string("cudaMallocHost: ") + cudaGetErrorString(ce));
  }
  for (int& t : s->ring_ticket) t = -1;
  for (cudaEvent_t& e : s->ring_ev) {
    ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      free_state(s);
      return fail(SEG_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
    }
  }
  for (cudaEvent_t& e : s->snap_ev) {
    ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      free_state(s);
      return fail(SEG_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
    }
  }
  std::memset(s->hctl, 0, sizeof(DevCtl));
  {
    std::vector<double> ones(kMaxCols, 1.0);
    ce = cudaMemcpy(s->ones, ones.data(), kMaxCols * sizeof(double), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      free_state(s);
      return fail(SEG_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(ce));
    }
  }
  // the step graph is built at the first graph-mode step (states that only
  // run inside batches never need one)
  seg_status st = SEG_OK;
  if (s->prec == SEG_MIXED_FP32) {
    fill_args<float>(s);
  } else {
    fill_args<double>(s);
  }
  if (st == SEG_OK) {
    const int* perm = p->perm;
    unsigned long long sd = (unsigned long long)seed;
    int kind = (int)init;
    st = launch_aux(s, s->ks.init_rng, (long long)p->n * s->ms, perm, sd, kind);
  }
  if (st == SEG_OK) {
    cudaError_t se = cudaStreamSynchronize(s->stream);
    if (se != cudaSuccess) st = fail(SEG_ERR_CUDA, std::string("init: ") + cudaGetErrorString(se));
  }
  if (st != SEG_OK) {
    free_state(s);
    return st;
  }
  s->pending = true;
  *out = s;
  return SEG_OK;
}

}  // extern "C"

long long segimpl::state_class_key(const seg_state* s) {
  return (long long)s->prec | (long long)s->lpr << 4 | (long long)s->p->ell_w << 12 | (long long)s->p->device << 20;
}

extern "C" {

seg_status seg_state_bytes(const seg_problem* p, int32_t m, uint64_t* bytes) {
  if (!p || !bytes) return fail(SEG_ERR_ARG, "problem or bytes is NULL");
  if (m < 1 || m > kMaxCols) return fail(SEG_ERR_ARG, "m must be in [1, 32]");
  int nsm = 0;
  SEG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
  const int vw = p->prec == SEG_MIXED_FP32 ? 4 : 2;
  int lpr = (m + vw - 1) / vw, pw = 1;
  while (pw < lpr) pw <<= 1;
  const uint64_t ms = (uint64_t)pw * vw, n = (uint64_t)p->n;
  // partial sums sized for every geometry the autotuner may pick
  const uint64_t grid = (uint64_t)std::min(kMaxGrid, kTuneWaves * kRowBlocksPerSM * nsm);
  const uint64_t grid_e = (uint64_t)std::min(kMaxGrid, kTuneWaves * kTriBlocksPerSM * nsm);
  const uint64_t vbytes = n * ms * vsize(p->prec);
  const uint64_t pbytes = partial_bytes((int)ms, (int)grid, (int)grid_e);
  *bytes = (p->prec == SEG_FP64 ? 9 : 8) * vbytes + sizeof(DevCtl) + pbytes + std::max<uint64_t>(8, n * m * 8) + 2 * kMaxCols * 8 +
           std::max<uint64_t>(4, n * 4) + std::max<uint64_t>(4, n);
  return SEG_OK;
}

void seg_state_destroy(seg_state* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  free_state(s);
}

seg_status seg_set_u(seg_state* s, const double* u, int32_t is_device) {
  if (!s || !u) return fail(SEG_ERR_ARG, "state or u is NULL");
  SEG_CUDA(cudaSetDevice(s->p->device));
  const double* src = u;
  if (!is_device) {
    SEG_CUDA(cudaMemcpyAsync(s->io, u, (size_t)s->p->n * s->m * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    src = s->io;
  }
  seg_status st = reset_ctl(s);
  if (st != SEG_OK) return st;
  // the first CG iteration multiplies the old search direction and its image
  // by beta = 0: clear them so that values left by a failed run cannot turn
  // into NaN; the solve of the first step starts from x = X (no correction)
  const size_t vbytes = (size_t)s->p->n * s->ms * vsize(s->prec);
  for (void* b : {s->Y, s->H0, s->H1, s->H2, s->P0, s->P1, s->Q})
    if (b) SEG_CUDA(cudaMemsetAsync(b, 0, vbytes, s->stream));
  const int* perm = s->p->perm;
  st = launch_aux(s, s->ks.scatter_in, (long long)s->p->n * s->ms, src, perm);
  if (st != SEG_OK) return st;
  SEG_CUDA(cudaStreamSynchronize(s->stream));
  s->pending = true;
  return SEG_OK;
}

seg_status seg_get_u(seg_state* s, double* u, int32_t is_device) {
  if (!s || !u) return fail(SEG_ERR_ARG, "state or u is NULL");
  SEG_CUDA(cudaSetDevice(s->p->device));
  seg_status st = ensure_norm(s);
  if (st != SEG_OK) return st;
  double* dst = is_device ? u : s->io;
  const int* iperm = s->p->iperm;
  st = launch_aux(s, s->ks.gather_out, (long long)s->p->n * s->m, dst, iperm);
  if (st != SEG_OK) return st;
  if (!is_device)
    SEG_CUDA(cudaMemcpyAsync(u, s->io, (size_t)s->p->n * s->m * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  st = sync_ctl(s);
  if (st != SEG_OK) return st;
  return (s->hctl->status & 2) ? status_from_ctl(*s->hctl) : SEG_OK;
}

// ------------------------------------------------------- checkpoint / resume

}  // extern "C"

namespace {

// Layout of a checkpoint: this header, the control block, then the state's
// vectors X, Y, H0, H1 (and H2 for float64 states) in internal row order.
struct CkptHeader {
  char magic[8];       // "SEGCKPT"
  int32_t version;     // kCkptVersion
  int32_t prec;        // seg_precision
  int64_t n;           // vertex rows
  int32_t m, ms;       // components, padded components
  double eps, tau;
  int32_t nvec;        // state-sized vectors after the control block
  int32_t pending;     // the normalisation of X is to be recomputed before it is read
  uint64_t vec_bytes;  // bytes of one vector
  uint64_t ctl_bytes;  // bytes of the control block
};
constexpr int32_t kCkptVersion = 1;
const char kCkptMagic[8] = {'S', 'E', 'G', 'C', 'K', 'P', 'T', 0};

int ckpt_vectors(const seg_state* s, void* const** out) {
  static thread_local void* v[5];
  v[0] = s->X;
  v[1] = s->Y;
  v[2] = s->H0;
  v[3] = s->H1;
  v[4] = s->H2;
  *out = v;
  return s->prec == SEG_FP64 ? 5 : 4;
}

uint64_t ckpt_bytes(const seg_state* s) {
  void* const* v;
  const int nv = ckpt_vectors(s, &v);
  return sizeof(CkptHeader) + sizeof(DevCtl) + (uint64_t)nv * (uint64_t)s->p->n * s->ms * vsize(s->prec);
}

}  // namespace

extern "C" {

seg_status seg_checkpoint_size(seg_state* s, uint64_t* bytes) {
  if (!s || !bytes) return fail(SEG_ERR_ARG, "state or bytes is NULL");
  *bytes = ckpt_bytes(s);
  return SEG_OK;
}

seg_status seg_get_checkpoint(seg_state* s, void* buf, uint64_t bytes) {
  if (!s || !buf) return fail(SEG_ERR_ARG, "state or buffer is NULL");
  if (bytes < ckpt_bytes(s)) return fail(SEG_ERR_ARG, "checkpoint buffer smaller than seg_checkpoint_size");
  SEG_CUDA(cudaSetDevice(s->p->device));
  SEG_CUDA(cudaStreamSynchronize(s->stream));
  void* const* v;
  const int nv = ckpt_vectors(s, &v);
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
  h.version = kCkptVersion;
  h.prec = (int32_t)s->prec;
  h.n = s->p->n;
  h.m = s->m;
  h.ms = s->ms;
  h.eps = s->eps;
  h.tau = s->p->tau;
  h.nvec = nv;
  h.pending = s->pending ? 1 : 0;
  h.vec_bytes = (uint64_t)s->p->n * s->ms * vsize(s->prec);
  h.ctl_bytes = sizeof(DevCtl);
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memcpy(out, &h, sizeof(h));
  out += sizeof(h);
  SEG_CUDA(cudaMemcpyAsync(out, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->stream));
  out += sizeof(DevCtl);
  for (int k = 0; k < nv; ++k) {
    SEG_CUDA(cudaMemcpyAsync(out, v[k], h.vec_bytes, cudaMemcpyDeviceToHost, s->stream));
    out += h.vec_bytes;
  }
  SEG_CUDA(cudaStreamSynchronize(s->stream));
  return SEG_OK;
}

seg_status seg_set_checkpoint(seg_state* s, const void* buf, uint64_t bytes) {
  if (!s || !buf) return fail(SEG_ERR_ARG, "state or buffer is NULL");
  if (bytes < sizeof(CkptHeader)) return fail(SEG_ERR_ARG, "checkpoint shorter than its header");
  CkptHeader h;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  std::memcpy(&h, in, sizeof(h));
  void* const* v;
  const int nv = ckpt_vectors(s, &v);
  const uint64_t vb = (uint64_t)s->p->n * s->ms * vsize(s->prec);
  if (std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0 || h.version != kCkptVersion)
    return fail(SEG_ERR_ARG, "not a checkpoint of this library version");
  if (h.prec != (int32_t)s->prec || h.n != s->p->n || h.m != s->m || h.ms != s->ms || h.nvec != nv ||
      h.vec_bytes != vb || h.ctl_bytes != sizeof(DevCtl))
    return fail(SEG_ERR_ARG, "checkpoint of another mesh size, m or precision");
  if (h.eps != s->eps || h.tau != s->p->tau) return fail(SEG_ERR_ARG, "checkpoint of another eps or tau");
  if (bytes < ckpt_bytes(s)) return fail(SEG_ERR_ARG, "checkpoint buffer shorter than its contents");
  SEG_CUDA(cudaSetDevice(s->p->device));
  SEG_CUDA(cudaStreamSynchronize(s->stream));
  in += sizeof(h);
  DevCtl c;
  std::memcpy(&c, in, sizeof(DevCtl));
  in += sizeof(DevCtl);
  for (unsigned int& t : c.counters) t = 0u;  // tickets are zero between launches
  std::memcpy(s->hctl, &c, sizeof(DevCtl));
  SEG_CUDA(cudaMemcpyAsync(s->ctl, s->hctl, sizeof(DevCtl), cudaMemcpyHostToDevice, s->stream));
  for (int k = 0; k < nv; ++k) {
    SEG_CUDA(cudaMemcpyAsync(v[k], in, vb, cudaMemcpyHostToDevice, s->stream));
    in += vb;
  }
  SEG_CUDA(cudaStreamSynchronize(s->stream));
  s->pending = h.pending != 0;
  s->peel_step = c.step;
  s->peel_it = c.cg_total;
  return SEG_OK;
}

seg_status seg_set_wait_limit(seg_state* s, int64_t ns) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  s->wait_ns = ns > 0 ? (unsigned long long)ns : kDefaultWaitNs;
  if (s->prec == SEG_MIXED_FP32)
    args_of<float>(s).wait_ns = s->wait_ns;
  else
    args_of<double>(s).wait_ns = s->wait_ns;
  retire_graph(s);  // the step graph holds the arguments it was built with
  return SEG_OK;
}

seg_status seg_set_wait_stall(seg_state* s, int32_t on) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  s->stall_waits = on != 0 ? 1 : 0;
  if (s->prec == SEG_MIXED_FP32)
    args_of<float>(s).stall_waits = s->stall_waits;
  else
    args_of<double>(s).stall_waits = s->stall_waits;
  retire_graph(s);
  return SEG_OK;
}

// ------------------------------------------------------------------- steps

}  // extern "C"

namespace {

// Start of a run of steps: remember the step count in stream order, and
// clear the sticky status bits of earlier calls; halted states stay halted.
seg_status begin_steps(seg_state* s) {
  SEG_CUDA(cudaSetDevice(s->p->device));
  SEG_CUDA(cudaMemcpyAsync(&s->ctl->step_mark, &s->ctl->step, sizeof(long long), cudaMemcpyDeviceToDevice,
                           s->stream));
  SEG_CUDA(cudaMemsetAsync(&s->ctl->status, 0, sizeof(int), s->stream));
  return SEG_OK;
}

seg_status enqueue_steps(seg_state* s, int64_t nsteps) {
  if (s->launch_mode == 0) {
    if (!s->exec) {
      const seg_status gs = s->prec == SEG_MIXED_FP32 ? build_graph_t<float>(s) : build_graph_t<double>(s);
      if (gs != SEG_OK) {
        drop_graph(s);
        return gs;
      }
    }
    for (int64_t k = 0; k < nsteps; ++k) SEG_CUDA(cudaGraphLaunch(s->exec, s->stream));
  } else {
    for (int64_t k = 0; k < nsteps; ++k) {
      seg_status st = direct_step(s);
      if (st != SEG_OK) return st;
    }
  }
  if (nsteps > 0) s->pending = true;
  return SEG_OK;
}

}  // namespace

extern "C" {

seg_status seg_step_async(seg_state* s, int64_t nsteps) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  if (nsteps < 0) return fail(SEG_ERR_ARG, "nsteps must be >= 0");
  seg_status st = begin_steps(s);
  if (st != SEG_OK) return st;
  return enqueue_steps(s, nsteps);
}

// Review the step graph's peel (CG iterations placed before its WHILE node)
// against the iterations per step since the last review: a pass after the
// solve has converged returns at once, an evaluation of the loop condition
// costs more, so the peel follows the mean rounded up.  It grows at once and
// shrinks only by two or more (no rebuild for a mean that hovers at an
// integer).  The graph is rebuilt at the next graph-mode step.  Called with
// the stream idle.
static void review_peel(seg_state* s, long long step, long long cg_total) {
  const long long ds = step - s->peel_step, di = cg_total - s->peel_it;
  if (ds < 0 || di < 0) {  // counters were reset (seg_set_u)
    s->peel_step = step;
    s->peel_it = cg_total;
    return;
  }
  if (ds < 3 || s->launch_mode != 0) return;
  const int target = std::min(kCgPeelMax, std::max(1, (int)std::ceil((double)di / (double)ds - 0.1)));
  if (target > s->cg_peel || target <= s->cg_peel - 2) {
    s->cg_peel = target;
    retire_graph(s);
  }
  s->peel_step = step;
  s->peel_it = cg_total;
}

seg_status seg_sync(seg_state* s, int64_t* steps_done) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  seg_status st = sync_ctl(s);
  if (st != SEG_OK) return st;
  drop_retired(s);
  review_peel(s, s->hctl->step, s->hctl->cg_total);
  if (steps_done) *steps_done = s->hctl->step - s->hctl->step_mark;
  return status_from_ctl(*s->hctl);
}

// Steps per chunk of a long synchronous run in graph mode.  The run is
// enqueued chunk by chunk, at most two chunks ahead of the device: after each
// chunk the step and CG iteration counters are copied to pinned memory, and
// once the chunk before has completed its counters review the graph's peel
// (a new graph is built for the next chunk if it changes; the device keeps
// working on the chunk in flight meanwhile).
constexpr int64_t kReviewChunk = 16;

seg_status seg_step(seg_state* s, int64_t nsteps, int64_t* steps_done) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  if (nsteps < 0) return fail(SEG_ERR_ARG, "nsteps must be >= 0");
  seg_status st = begin_steps(s);
  if (st != SEG_OK) return st;
  if (s->launch_mode != 0 || nsteps < 4 * kReviewChunk) {
    st = enqueue_steps(s, nsteps);
    if (st != SEG_OK) return st;
    return seg_sync(s, steps_done);
  }
  int slot = 0;
  bool have_prev = false;
  for (int64_t left = nsteps; left > 0;) {
    const int64_t n = std::min(left, kReviewChunk);
    st = enqueue_steps(s, n);
    if (st != SEG_OK) return st;
    left -= n;
    long long* snap = s->hsnap + 2 * slot;
    SEG_CUDA(cudaMemcpyAsync(snap, &s->ctl->step, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    SEG_CUDA(cudaMemcpyAsync(snap + 1, &s->ctl->cg_total, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    SEG_CUDA(cudaEventRecord(s->snap_ev[slot], s->stream));
    if (have_prev && left > 0) {
      const int prev = slot ^ 1;
      SEG_CUDA(cudaEventSynchronize(s->snap_ev[prev]));
      review_peel(s, s->hsnap[2 * prev], s->hsnap[2 * prev + 1]);
    }
    have_prev = true;
    slot ^= 1;
  }
  return seg_sync(s, steps_done);
}

seg_status seg_substep(seg_state* s, int32_t stage) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  if (stage < 1 || stage > 3) return fail(SEG_ERR_ARG, "stage must be 1, 2 or 3");
  SEG_CUDA(cudaSetDevice(s->p->device));
  seg_status st = SEG_OK;
  if (stage == 1) {
    const bool keep_scale = !s->pending;
    if (keep_scale)
      SEG_CUDA(cudaMemcpyAsync(s->scale_backup, s->ctl->inv_n, kMaxCols * sizeof(double), cudaMemcpyDeviceToDevice,
                               s->stream));
    SEG_CUDA(cudaMemsetAsync(&s->ctl->status, 0, sizeof(int), s->stream));
    st = launch_row(s, s->ks.start, Launch());
    if (st != SEG_OK) return st;
    s->pending = false;
    st = sync_ctl(s);
    if (st != SEG_OK) return st;
    while (s->hctl->cont) {
      if ((st = launch_row(s, s->ks.cg_a, Launch())) != SEG_OK) return st;
      if ((st = launch_row(s, s->ks.cg_b, Launch())) != SEG_OK) return st;
      if ((st = sync_ctl(s)) != SEG_OK) return st;
    }
    Launch l;
    l.apply_x = 1;
    if ((st = launch_row(s, s->ks.finish, l)) != SEG_OK) return st;
    if (keep_scale)
      SEG_CUDA(cudaMemcpyAsync(s->ctl->inv_n, s->scale_backup, kMaxCols * sizeof(double), cudaMemcpyDeviceToDevice,
                               s->stream));
  } else if (stage == 2) {
    if ((st = ensure_norm(s)) != SEG_OK) return st;
    Launch l;
    l.apply_ode = 1;
    if ((st = launch_row(s, s->ks.finish, l)) != SEG_OK) return st;
    SEG_CUDA(cudaMemcpyAsync(s->ctl->inv_n, s->ones, kMaxCols * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    s->pending = false;
  } else {
    s->pending = true;
    if ((st = ensure_norm(s)) != SEG_OK) return st;
  }
  st = sync_ctl(s);
  if (st != SEG_OK) return st;
  return status_from_ctl(*s->hctl);
}

// ---------------------------------------------------------------- batches

}  // extern "C"

struct seg_batch {
  std::vector<seg_state*> members;
  seg_precision prec = SEG_FP64;
  KernelSet ks{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int* amap = nullptr;  // device [kMaxBatch]: members iterating in the current CG iteration
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int peel = 0;  // CG iterations of the graph ahead of its loop node (0: the members' largest)
  // graphs replaced while launches of them may still be in flight
  std::vector<std::pair<cudaGraph_t, cudaGraphExec_t>> retired;
  long long* hsnap = nullptr;  // pinned: 2 slots x members x (step, cg_total)
  cudaEvent_t snap_ev[2] = {nullptr, nullptr};
  std::vector<long long> mark_step, mark_it;  // members' counters at the last peel review
  // persistent mode: every seg_batch_step call is one cooperative launch
  bool persistent = false;
  PersistCtl* pc = nullptr;  // device: grid barrier and phase decisions
  int persist_grid = 0;      // resident blocks of the persistent kernel
  unsigned persist_smem = 0;
};

namespace {

template <typename T>
cudaError_t add_batch_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                           void* fn, const BatchArgs<T>& b, int grid, int threads, unsigned smem) {
  BatchArgs<T> copy = b;
  void* args[] = {&copy};
  cudaKernelNodeParams kp{};
  kp.func = fn;
  kp.gridDim = dim3(grid > 0 ? grid : 1);
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = smem;
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

// The batch's step graph: the passes of Algorithm 2.2 as in the state's own
// graph, each one launch for every member.  Member i runs each pass on the
// virtual blocks of its own launch geometry (so its results are bitwise
// those of the member stepped alone); the physical grid of a pass is the
// members' virtual blocks together, at most the blocks resident at once.
template <typename T>
seg_status build_batch_t(seg_batch* b) {
  const int n = (int)b->members.size();
  std::vector<KArgs<T>> tab(n);
  BatchArgs<T> rows[4] = {}, tris{}, vote{};
  int nsm = 0;
  SEG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->members[0]->p->device));
  int phys[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    seg_state* s = b->members[i];
    Launch l;
    l.ignore_halt = 0;
    l.apply_x = 1;
    l.apply_ode = 1;
    l.count_step = 1;
    tab[i] = make_args<T>(s, l);
    for (int k = 0; k < 4; ++k) {
      rows[k].vg[i] = s->grid[k];
      phys[k] += s->grid[k];
    }
    tris.vg[i] = s->grid_e;
    phys[4] += s->grid_e;
  }
  for (int k = 0; k < 4; ++k)
    phys[k] = std::min(phys[k], nsm * (k == kPassStart ? kStartBlocksPerSM : kRowBlocksPerSM));
  phys[4] = std::min(phys[4], nsm * kTriBlocksPerSM);
  rows[kPassStart].map = kMapAll;
  rows[kPassCgA].map = kMapCgA;
  rows[kPassCgB].map = kMapCgB;
  rows[kPassFinish].map = kMapAll;
  tris.map = kMapAll;

  SEG_CUDA(cudaGraphCreate(&b->graph, 0));
  SEG_CUDA(cudaGraphConditionalHandleCreate(&b->cond, b->graph, 0, cudaGraphCondAssignDefault));
  for (BatchArgs<T>* x : {&rows[0], &rows[1], &rows[2], &rows[3], &tris, &vote}) {
    for (int i = 0; i < n; ++i) x->tab[i] = tab[i];
    x->ninst = n;
    x->amap = b->amap;
    x->cond = (unsigned long long)b->cond;
  }
  cudaGraphNode_t n_start, n_energy, n_vote0, n_loop, n_a, n_b, n_vote, n_fin;
  SEG_CUDA(add_batch_node<T>(&n_start, b->graph, nullptr, 0, b->ks.b_start, rows[kPassStart], phys[kPassStart],
                             kBlockThreads, b->ks.smem_start));
  SEG_CUDA(add_batch_node<T>(&n_energy, b->graph, &n_start, 1, b->ks.b_energy_check, tris, phys[4], kBlockThreads,
                             0));
  // as in the single-state graph: the first CG iterations (at first the
  // largest peel count of the members, then reviewed while stepping) as
  // plain nodes, then the vote and the loop
  if (b->peel <= 0)
    for (seg_state* m : b->members) b->peel = std::max(b->peel, m->cg_peel);
  const int peel = b->peel;
  SEG_CUDA(add_batch_node<T>(&n_a, b->graph, &n_energy, 1, b->ks.b_cg_a, rows[kPassCgA], phys[kPassCgA],
                             kBlockThreads, b->ks.smem_cg_a));
  cudaGraphNode_t last = n_a;
  for (int u = 1; u < peel; ++u) {
    SEG_CUDA(add_batch_node<T>(&n_b, b->graph, &last, 1, b->ks.b_cg_b, rows[kPassCgB], phys[kPassCgB],
                               kBlockThreads, 0));
    SEG_CUDA(add_batch_node<T>(&n_a, b->graph, &n_b, 1, b->ks.b_cg_a, rows[kPassCgA], phys[kPassCgA],
                               kBlockThreads, b->ks.smem_cg_a));
    last = n_a;
  }
  SEG_CUDA(add_batch_node<T>(&n_vote0, b->graph, &last, 1, b->ks.b_vote, vote, 1, kMaxBatch, 0));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = b->cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  SEG_CUDA(cudaGraphAddNode(&n_loop, b->graph, &n_vote0, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaGraphNode_t prev = nullptr;
  for (int u = 0; u < kCgUnroll; ++u) {
    SEG_CUDA(add_batch_node<T>(&n_b, body, prev ? &prev : nullptr, prev ? 1 : 0, b->ks.b_cg_b, rows[kPassCgB],
                               phys[kPassCgB], kBlockThreads, 0));
    SEG_CUDA(add_batch_node<T>(&n_a, body, &n_b, 1, b->ks.b_cg_a, rows[kPassCgA], phys[kPassCgA], kBlockThreads,
                               b->ks.smem_cg_a));
    prev = n_a;
  }
  SEG_CUDA(add_batch_node<T>(&n_vote, body, &n_a, 1, b->ks.b_vote, vote, 1, kMaxBatch, 0));
  SEG_CUDA(add_batch_node<T>(&n_fin, b->graph, &n_loop, 1, b->ks.b_finish, rows[kPassFinish], phys[kPassFinish],
                             kBlockThreads, 0));
  SEG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return SEG_OK;
}

}  // namespace

extern "C" {

seg_status seg_batch_create(seg_state* const* states, int32_t n, void* cuda_stream, seg_batch** out) {
  if (!out) return fail(SEG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!states || n < 1 || n > kMaxBatch) return fail(SEG_ERR_ARG, "a batch holds 1 to 32 states");
  seg_state* s0 = states[0];
  if (!s0) return fail(SEG_ERR_ARG, "state is NULL");
  for (int i = 0; i < n; ++i) {
    seg_state* s = states[i];
    if (!s) return fail(SEG_ERR_ARG, "state is NULL");
    for (int j = 0; j < i; ++j)
      if (states[j] == s) return fail(SEG_ERR_ARG, "a state appears twice in the batch");
    if (s->prec != s0->prec || s->lpr != s0->lpr || s->p->ell_w != s0->p->ell_w || s->p->device != s0->p->device)
      return fail(SEG_ERR_ARG,
                  "batch members must share precision, padded component count class, row width and device");
  }
  SEG_CUDA(cudaSetDevice(s0->p->device));
  seg_batch* b = new (std::nothrow) seg_batch;
  if (!b) return fail(SEG_ERR_NO_MEMORY, "host allocation failed");
  b->members.assign(states, states + n);
  b->prec = s0->prec;
  b->ks = s0->ks;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  seg_status st = e == cudaSuccess ? SEG_OK : fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  // members' pending work on their own streams must be done first
  for (int i = 0; i < n && st == SEG_OK; ++i) {
    e = cudaStreamSynchronize(states[i]->stream);
    if (e != cudaSuccess) st = fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  }
  if (st == SEG_OK) {
    e = cudaMalloc((void**)&b->amap, kMaxBatch * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->amap, 0, kMaxBatch * sizeof(int));
    if (e != cudaSuccess) st = fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  }
  if (st == SEG_OK) {
    e = cudaMallocHost((void**)&b->hsnap, 4 * (size_t)n * sizeof(long long));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->snap_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) st = fail(SEG_ERR_CUDA, cudaGetErrorString(e));
  }
  if (st == SEG_OK) {
    // members' counters as of now (their streams are idle) start the first review
    b->mark_step.assign(n, 0);
    b->mark_it.assign(n, 0);
    for (int i = 0; i < n && st == SEG_OK; ++i) {
      st = sync_ctl(states[i]);
      if (st == SEG_OK) {
        b->mark_step[i] = states[i]->hctl->step;
        b->mark_it[i] = states[i]->hctl->cg_total;
      }
    }
  }
  if (st == SEG_OK) st = b->prec == SEG_MIXED_FP32 ? build_batch_t<float>(b) : build_batch_t<double>(b);
  if (st != SEG_OK) {
    seg_batch_destroy(b);
    return st;
  }
  *out = b;
  return SEG_OK;
}

}  // extern "C"

namespace {

seg_status begin_batch_steps(seg_batch* b) {
  SEG_CUDA(cudaSetDevice(b->members[0]->p->device));
  for (seg_state* s : b->members) {
    SEG_CUDA(cudaMemcpyAsync(&s->ctl->step_mark, &s->ctl->step, sizeof(long long), cudaMemcpyDeviceToDevice,
                             b->stream));
    SEG_CUDA(cudaMemsetAsync(&s->ctl->status, 0, sizeof(int), b->stream));
  }
  return SEG_OK;
}

template <typename T>
seg_status launch_persistent_t(seg_batch* b, int64_t nsteps) {
  PersistArgs<T> pa{};
  pa.ninst = (int)b->members.size();
  for (int i = 0; i < pa.ninst; ++i) {
    seg_state* s = b->members[i];
    Launch l;
    l.ignore_halt = 0;
    l.apply_x = 1;
    l.apply_ode = 1;
    l.count_step = 1;
    pa.tab[i] = make_args<T>(s, l);
    for (int k = 0; k < 4; ++k) pa.vg[k][i] = s->grid[k];
    pa.vg[4][i] = s->grid_e;
  }
  pa.pc = b->pc;
  pa.nsteps = nsteps;
  pa.wait_ns = kDefaultWaitNs;
  SEG_CUDA(cudaMemsetAsync(b->pc, 0, sizeof(PersistCtl), b->stream));
  void* args[] = {&pa};
  SEG_CUDA(cudaLaunchCooperativeKernel(b->ks.persist, dim3(b->persist_grid), dim3(kBlockThreads), args,
                                       b->persist_smem, b->stream));
  return SEG_OK;
}

seg_status enqueue_batch_steps(seg_batch* b, int64_t nsteps) {
  if (b->persistent) {
    if (nsteps > 0) {
      const seg_status st =
          b->prec == SEG_MIXED_FP32 ? launch_persistent_t<float>(b, nsteps) : launch_persistent_t<double>(b, nsteps);
      if (st != SEG_OK) return st;
      for (seg_state* s : b->members) s->pending = true;
    }
    return SEG_OK;
  }
  if (!b->exec) {
    const seg_status gs = b->prec == SEG_MIXED_FP32 ? build_batch_t<float>(b) : build_batch_t<double>(b);
    if (gs != SEG_OK) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      return gs;
    }
  }
  for (int64_t k = 0; k < nsteps; ++k) SEG_CUDA(cudaGraphLaunch(b->exec, b->stream));
  if (nsteps > 0)
    for (seg_state* s : b->members) s->pending = true;
  return SEG_OK;
}

void drop_batch_retired(seg_batch* b) {
  for (auto& r : b->retired) {
    if (r.second) cudaGraphExecDestroy(r.second);
    if (r.first) cudaGraphDestroy(r.first);
  }
  b->retired.clear();
}

// The batch's graph runs as many CG iterations per step as its slowest
// member: review its peel against the largest mean iterations per step of
// the members since the last review (the same rule as review_peel; members
// that took no step, e.g. stopped ones, are left out).  snap holds the
// members' (step, cg_total) pairs.
void review_batch_peel(seg_batch* b, const long long* snap) {
  const size_t n = b->members.size();
  double worst = 0.0;
  long long most = 0;
  for (size_t i = 0; i < n; ++i) {
    const long long ds = snap[2 * i] - b->mark_step[i], di = snap[2 * i + 1] - b->mark_it[i];
    if (ds > 0 && di >= 0) worst = std::max(worst, (double)di / (double)ds);
    most = std::max(most, ds);
  }
  if (most < 3) return;
  const int target = std::min(kCgPeelMax, std::max(1, (int)std::ceil(worst - 0.1)));
  if (target > b->peel || target <= b->peel - 2) {
    b->peel = target;
    if (b->exec || b->graph) b->retired.emplace_back(b->graph, b->exec);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  for (size_t i = 0; i < n; ++i) {
    b->mark_step[i] = snap[2 * i];
    b->mark_it[i] = snap[2 * i + 1];
  }
}

}  // namespace

extern "C" {

seg_status seg_batch_step_async(seg_batch* b, int64_t nsteps) {
  if (!b) return fail(SEG_ERR_ARG, "batch is NULL");
  if (nsteps < 0) return fail(SEG_ERR_ARG, "nsteps must be >= 0");
  seg_status st = begin_batch_steps(b);
  if (st != SEG_OK) return st;
  return enqueue_batch_steps(b, nsteps);
}

seg_status seg_batch_sync(seg_batch* b) {
  if (!b) return fail(SEG_ERR_ARG, "batch is NULL");
  for (seg_state* s : b->members)
    SEG_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, b->stream));
  SEG_CUDA(cudaStreamSynchronize(b->stream));
  drop_batch_retired(b);
  for (seg_state* s : b->members) {
    seg_status st = status_from_ctl(*s->hctl);
    if (st != SEG_OK) return st;
  }
  return SEG_OK;
}

// As seg_step: a run of 64 or more steps is enqueued in chunks of 16, at
// most two ahead of the device, and the graph's peel is reviewed between
// chunks from the members' counters.
seg_status seg_batch_step(seg_batch* b, int64_t nsteps) {
  if (!b) return fail(SEG_ERR_ARG, "batch is NULL");
  if (nsteps < 0) return fail(SEG_ERR_ARG, "nsteps must be >= 0");
  seg_status st = begin_batch_steps(b);
  if (st != SEG_OK) return st;
  if (nsteps < 4 * kReviewChunk || b->persistent) {  // (a persistent batch: one launch)
    st = enqueue_batch_steps(b, nsteps);
    if (st != SEG_OK) return st;
    return seg_batch_sync(b);
  }
  const size_t n = b->members.size();
  int slot = 0;
  bool have_prev = false;
  for (int64_t left = nsteps; left > 0;) {
    const int64_t c = std::min(left, kReviewChunk);
    st = enqueue_batch_steps(b, c);
    if (st != SEG_OK) return st;
    left -= c;
    long long* snap = b->hsnap + 2 * n * slot;
    for (size_t i = 0; i < n; ++i) {
      seg_state* s = b->members[i];
      SEG_CUDA(cudaMemcpyAsync(snap + 2 * i, &s->ctl->step, sizeof(long long), cudaMemcpyDeviceToHost, b->stream));
      SEG_CUDA(cudaMemcpyAsync(snap + 2 * i + 1, &s->ctl->cg_total, sizeof(long long), cudaMemcpyDeviceToHost,
                               b->stream));
    }
    SEG_CUDA(cudaEventRecord(b->snap_ev[slot], b->stream));
    if (have_prev && left > 0) {
      const int prev = slot ^ 1;
      SEG_CUDA(cudaEventSynchronize(b->snap_ev[prev]));
      review_batch_peel(b, b->hsnap + 2 * n * prev);
    }
    have_prev = true;
    slot ^= 1;
  }
  return seg_batch_sync(b);
}

void seg_batch_destroy(seg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_batch_retired(b);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->amap) cudaFree(b->amap);
  if (b->pc) cudaFree(b->pc);
  if (b->hsnap) cudaFreeHost(b->hsnap);
  for (cudaEvent_t e : b->snap_ev)
    if (e) cudaEventDestroy(e);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

seg_status seg_batch_set_persistent(seg_batch* b, int32_t on) {
  if (!b) return fail(SEG_ERR_ARG, "batch is NULL");
  if (!on) {
    b->persistent = false;
    return SEG_OK;
  }
  const int dev = b->members[0]->p->device;
  SEG_CUDA(cudaSetDevice(dev));
  int coop = 0, nsm = 0;
  SEG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  SEG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (!coop) return fail(SEG_ERR_UNSUPPORTED, "the device does not support cooperative launches");
  const unsigned smem = std::max(b->ks.smem_start, b->ks.smem_cg_a);
  SEG_CUDA(cudaFuncSetAttribute(b->ks.persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  SEG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, b->ks.persist, kBlockThreads, smem));
  if (occ < 1) return fail(SEG_ERR_UNSUPPORTED, "the persistent kernel does not fit on a multiprocessor");
  if (!b->pc) {
    cudaError_t e = cudaMalloc((void**)&b->pc, sizeof(PersistCtl));
    if (e == cudaSuccess) e = cudaMemset(b->pc, 0, sizeof(PersistCtl));
    if (e != cudaSuccess) {
      if (b->pc) cudaFree(b->pc);
      b->pc = nullptr;
      return fail(SEG_ERR_NO_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  b->persist_smem = smem;
  b->persist_grid = occ * nsm;
  b->persistent = true;
  return SEG_OK;
}

// ---------------------------------------------------------------- outputs

// S_eps (and, with per_component, the coupling integrals) of the
// renormalised current state.
static seg_status evaluate_energy(seg_state* s, bool per_component) {
  SEG_CUDA(cudaSetDevice(s->p->device));
  s->pending = true;
  seg_status st = ensure_norm(s);
  if (st != SEG_OK) return st;
  Launch l;
  l.force = 1;
  st = launch_row(s, per_component ? s->ks.energy : s->ks.energy_check, l);
  if (st != SEG_OK) return st;
  return sync_ctl(s);
}

seg_status seg_energy(seg_state* s, double* total, double* functional, double* dirichlet, double* s_eps) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  seg_status st = evaluate_energy(s, false);
  if (st != SEG_OK) return st;
  const DevCtl& c = *s->hctl;
  if (total) *total = c.e_total;
  if (functional) *functional = 0.5 * c.e_dir + c.e_s;
  if (dirichlet) *dirichlet = c.e_dir;
  if (s_eps) *s_eps = c.e_s;
  if (!std::isfinite(c.e_total)) return fail(SEG_ERR_NONFINITE, "energy is not finite");
  return (c.status & 2) ? status_from_ctl(c) : SEG_OK;
}

seg_status seg_eigenvalue_estimates(seg_state* s, double* lambda, double* lambda_cl) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  seg_status st = evaluate_energy(s, true);
  if (st != SEG_OK) return st;
  const DevCtl& c = *s->hctl;
  for (int i = 0; i < s->m; ++i) {
    if (lambda) lambda[i] = c.lam[i];
    if (lambda_cl) lambda_cl[i] = c.lam[i] + 2.0 * c.coup[i] / (s->eps * s->eps);
  }
  return (c.status & 2) ? status_from_ctl(c) : SEG_OK;
}

seg_status seg_energy_p(seg_state* s, double p, double* e_p) {
  if (!s || !e_p) return fail(SEG_ERR_ARG, "state or output is NULL");
  if (!(p >= 1.0)) return fail(SEG_ERR_ARG, "p must be >= 1 (or +inf)");
  seg_status st = evaluate_energy(s, false);
  if (st != SEG_OK) return st;
  const DevCtl& c = *s->hctl;
  if (std::isinf(p)) {
    double mx = c.lam[0];
    for (int i = 1; i < s->m; ++i) mx = std::max(mx, c.lam[i]);
    *e_p = mx;
  } else {
    // scaled by the largest value so that lambda^p cannot overflow
    double top = c.lam[0];
    for (int i = 1; i < s->m; ++i) top = std::max(top, c.lam[i]);
    double acc = 0.0;
    for (int i = 0; i < s->m; ++i) acc += top > 0.0 ? std::pow(c.lam[i] / top, p) : 0.0;
    *e_p = top > 0.0 ? top * std::pow(acc / s->m, 1.0 / p) : 0.0;
  }
  return (c.status & 2) ? status_from_ctl(c) : SEG_OK;
}

seg_status seg_prolong(seg_state* coarse, seg_state* fine, const int32_t* parents) {
  if (!coarse || !fine || !parents) return fail(SEG_ERR_ARG, "coarse, fine or parents is NULL");
  if (coarse->m != fine->m) return fail(SEG_ERR_ARG, "coarse and fine states need the same m");
  if (coarse->p->device != fine->p->device) return fail(SEG_ERR_ARG, "states live on different devices");
  const int64_t nc = coarse->p->n, nf = fine->p->n;
  for (int64_t k = 0; k < 2 * nf; ++k)
    if (parents[k] < 0 || parents[k] >= nc) return fail(SEG_ERR_ARG, "parent index out of range");
  SEG_CUDA(cudaSetDevice(fine->p->device));
  const int m = fine->m;
  double* uc = nullptr;
  double* uf = nullptr;
  int32_t* par = nullptr;
  cudaError_t ce = cudaMalloc(&uc, (size_t)nc * m * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMalloc(&uf, (size_t)nf * m * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMalloc(&par, (size_t)nf * 2 * sizeof(int32_t));
  seg_status st = SEG_OK;
  if (ce != cudaSuccess) st = fail(SEG_ERR_NO_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
  if (st == SEG_OK) st = seg_get_u(coarse, uc, 1);  // caller numbering, synchronised
  if (st == SEG_OK) {
    ce = cudaMemcpyAsync(par, parents, (size_t)nf * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, fine->stream);
    if (ce == cudaSuccess) {
      const long long total = (long long)nf * m;
      k_prolong<<<(unsigned)((total + 255) / 256), 256, 0, fine->stream>>>(uc, par, uf, nf, m);
      ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) st = fail(SEG_ERR_CUDA, std::string("prolongation: ") + cudaGetErrorString(ce));
  }
  if (st == SEG_OK) st = seg_set_u(fine, uf, 1);  // synchronises fine's stream
  cudaFree(uc);
  cudaFree(uf);
  cudaFree(par);
  return st;
}

seg_status seg_continue(seg_state* coarse, const seg_mesh* coarse_mesh, const seg_surface* surf, double eps_next,
                        double tau_next, const seg_params* opt, seg_mesh** fine_mesh, seg_problem** fine_problem,
                        seg_state** fine_state) {
  if (!fine_mesh || !fine_problem || !fine_state) return fail(SEG_ERR_ARG, "an output is NULL");
  *fine_mesh = nullptr;
  *fine_problem = nullptr;
  *fine_state = nullptr;
  if (!coarse || !coarse_mesh || !surf) return fail(SEG_ERR_ARG, "coarse state, mesh or surface is NULL");
  if (coarse_mesh->h.n != coarse->p->n) return fail(SEG_ERR_ARG, "coarse mesh does not match the coarse state");
  seg_mesh* fm = nullptr;
  seg_problem* fp = nullptr;
  seg_state* fs = nullptr;
  std::vector<int32_t> parents(2 * (coarse_mesh->h.n + 3 * coarse_mesh->h.f));
  seg_status st = seg_mesh_refine(coarse_mesh, surf, &fm, parents.data());
  if (st == SEG_OK) st = seg_assemble_ex(fm, tau_next, coarse->prec, coarse->p->flags, &fp);
  if (st == SEG_OK) st = seg_state_create(fp, coarse->m, eps_next, SEG_INIT_UNIFORM, 0, opt, nullptr, &fs);
  if (st == SEG_OK) st = seg_prolong(coarse, fs, parents.data());
  if (st != SEG_OK) {
    seg_state_destroy(fs);
    seg_problem_destroy(fp);
    seg_mesh_destroy(fm);
    return st;
  }
  *fine_mesh = fm;
  *fine_problem = fp;
  *fine_state = fs;
  return SEG_OK;
}

seg_status seg_labels(seg_state* s, int32_t* argmax, uint8_t* v_positive) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  SEG_CUDA(cudaSetDevice(s->p->device));
  seg_status st = ensure_norm(s);
  if (st != SEG_OK) return st;
  int* am = s->am;
  unsigned char* vp = s->vp;
  const int* iperm = s->p->iperm;
  st = launch_aux(s, s->ks.labels, s->p->n, am, vp, iperm);
  if (st != SEG_OK) return st;
  if (argmax) SEG_CUDA(cudaMemcpyAsync(argmax, s->am, (size_t)s->p->n * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  if (v_positive) SEG_CUDA(cudaMemcpyAsync(v_positive, s->vp, (size_t)s->p->n, cudaMemcpyDeviceToHost, s->stream));
  return sync_ctl(s);
}

}  // extern "C"

namespace {

void stats_of(const seg_state* s, const DevCtl& c, seg_stats* out) {
  out->steps = c.step;
  out->cg_iterations = c.cg_total;
  out->cg_last = c.cg_last;
  out->cg_max = c.cg_max;
  out->converged = c.halted == 1 ? 1 : 0;
  out->status_bits = c.status;
  out->last_check_total = c.e_prev;
  out->checks = c.checks;
  out->kernel_launches = (int64_t)c.launches;
  out->graph_peel = s->cg_peel;
  out->reserved = 0;
}

}  // namespace

extern "C" {

seg_status seg_get_stats(seg_state* s, seg_stats* out) {
  if (!s || !out) return fail(SEG_ERR_ARG, "state or out is NULL");
  SEG_CUDA(cudaSetDevice(s->p->device));
  seg_status st = sync_ctl(s);
  if (st != SEG_OK) return st;
  stats_of(s, *s->hctl, out);
  return SEG_OK;
}

seg_status seg_stats_enqueue(seg_state* s, int32_t* ticket) {
  if (!s || !ticket) return fail(SEG_ERR_ARG, "state or ticket is NULL");
  SEG_CUDA(cudaSetDevice(s->p->device));
  const int t = s->ring_next;
  const int slot = t % SEG_STATS_RING;
  SEG_CUDA(cudaMemcpyAsync(s->hring + slot, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s->stream));
  SEG_CUDA(cudaEventRecord(s->ring_ev[slot], s->stream));
  s->ring_ticket[slot] = t;
  s->ring_next = t == 0x7fffffff ? 0 : t + 1;
  *ticket = t;
  return SEG_OK;
}

seg_status seg_stats_wait(seg_state* s, int32_t ticket, seg_stats* out) {
  if (!s || !out) return fail(SEG_ERR_ARG, "state or out is NULL");
  if (ticket < 0 || s->ring_ticket[ticket % SEG_STATS_RING] != ticket)
    return fail(SEG_ERR_ARG, "unknown or overwritten statistics ticket");
  const int slot = ticket % SEG_STATS_RING;
  SEG_CUDA(cudaEventSynchronize(s->ring_ev[slot]));
  stats_of(s, s->hring[slot], out);
  return SEG_OK;
}

// -------------------------------------------------------------- diagnostics

seg_status seg_time_kernel(seg_state* s, int32_t which, int32_t reps, double* ms_per_launch) {
  if (!s || !ms_per_launch) return fail(SEG_ERR_ARG, "state or output is NULL");
  if (which < 0 || which > 9 || reps < 1) return fail(SEG_ERR_ARG, "which must be 0..9 and reps >= 1");
  SEG_CUDA(cudaSetDevice(s->p->device));
  seg_status st = time_launches(s, which, reps, ms_per_launch);
  s->pending = true;
  return st;
}

seg_status seg_autotune(seg_state* s, int32_t reps, seg_tune_result* out) {
  if (!s || !out) return fail(SEG_ERR_ARG, "state or out is NULL");
  if (reps < 1) reps = 10;
  std::memset(out, 0, sizeof(*out));
  SEG_CUDA(cudaSetDevice(s->p->device));
  int nsm = 0;
  SEG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->p->device));
  seg_status st = sync_ctl(s);
  if (st != SEG_OK) return st;
  // CG iterations per step so far (the weight of the two CG passes)
  const double k = s->hctl->step > 0 ? (double)s->hctl->cg_total / (double)s->hctl->step : 8.0;
  // CG pass B launches per step: none in a solve of one iteration (it ends
  // in CG pass A), j in a solve of j >= 2 (mixing counts of 1 and 2 below 2)
  const double kb = k >= 2.0 ? k : std::max(0.0, 2.0 * (k - 1.0));
  // save the data the timing launches overwrite: X, Y, H0, H1 and the control block;
  // Z, P and Q are rewritten by every step before they are read (the first
  // CG pass of a solve does not read P)
  const size_t vbytes = (size_t)s->p->n * s->ms * vsize(s->prec);
  void* saved_x = nullptr;  // X, Y and the history slots
  DevCtl* saved_ctl = nullptr;
  std::vector<void*> keep = {s->X, s->Y, s->H0, s->H1};
  if (s->H2) keep.push_back(s->H2);
  const size_t nkeep = keep.size();
  cudaError_t ce = cudaMalloc(&saved_x, nkeep * vbytes);
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&saved_ctl, sizeof(DevCtl));
  if (ce != cudaSuccess) {
    cudaFree(saved_x);
    return fail(SEG_ERR_NO_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
  }
  const bool pending = s->pending;
  int grid0[4];
  for (int w = 0; w < 4; ++w) grid0[w] = s->grid[w];
  const int grid_e0 = s->grid_e;
  ce = cudaSuccess;
  for (size_t b = 0; b < nkeep && ce == cudaSuccess; ++b)
    ce = cudaMemcpyAsync((char*)saved_x + b * vbytes, keep[b], vbytes, cudaMemcpyDeviceToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(saved_ctl, s->ctl, sizeof(DevCtl), cudaMemcpyDeviceToDevice, s->stream);
  if (ce != cudaSuccess) st = fail(SEG_ERR_CUDA, std::string("save: ") + cudaGetErrorString(ce));
  // candidate row grids: 1 .. kRowBlocksPerSM blocks per SM (one wave), and
  // 2 .. kTuneWaves waves of them (the hardware hands out the later blocks as
  // earlier ones finish), at most one block per 256 rows; triangle grids
  // likewise with kTriBlocksPerSM.  Each pass gets its own grid.
  std::vector<int> rows_c, tris_c;
  const int64_t n_cap = std::max<int64_t>(1, (s->p->n + 255) / 256);
  const int64_t f_cap = std::max<int64_t>(1, (s->p->f + 1023) / 1024);
  for (int b = 1; b <= kRowBlocksPerSM; ++b) rows_c.push_back((int)std::min<int64_t>((int64_t)b * nsm, n_cap));
  for (int b = 1; b <= kTriBlocksPerSM; ++b) tris_c.push_back((int)std::min<int64_t>((int64_t)b * nsm, f_cap));
  for (int w = 2; w <= kTuneWaves; w *= 2) {
    rows_c.push_back((int)std::min<int64_t>((int64_t)w * kRowBlocksPerSM * nsm, n_cap));
    tris_c.push_back((int)std::min<int64_t>((int64_t)w * kTriBlocksPerSM * nsm, f_cap));
  }
  for (int w = 0; w < 4; ++w) rows_c.push_back(grid0[w]);
  tris_c.push_back(grid_e0);
  for (auto* v : {&rows_c, &tris_c}) {
    std::sort(v->begin(), v->end());
    v->erase(std::unique(v->begin(), v->end()), v->end());
  }
  int best[4];
  double best_t[4];
  for (int w = 0; w < 4; ++w) {
    best[w] = grid0[w];
    best_t[w] = 1e300;
  }
  int best_e = grid_e0;
  double best_e_ms = 1e300;
  for (size_t c = 0; c < rows_c.size() && st == SEG_OK; ++c) {
    const int g = rows_c[c];
    if (g > s->grid_cap) continue;
    for (int w = 0; w < 4; ++w) s->grid[w] = g;
    double t[4] = {0, 0, 0, 0};
    for (int w = 0; w < 4 && st == SEG_OK; ++w) st = time_launches(s, w, reps, &t[w]);
    double t_odd = 0;  // CG pass A alternates between its even and odd form
    if (st == SEG_OK) st = time_launches(s, 6, reps, &t_odd);
    if (st != SEG_OK) break;
    t[1] = 0.5 * (t[1] + t_odd);
    const double model = t[0] + k * t[1] + kb * t[2] + t[3];
    if (out->n_candidates < SEG_TUNE_MAX) {
      out->cand_grid[out->n_candidates] = g;
      out->cand_ms[out->n_candidates] = model;
      out->n_candidates += 1;
    }
    for (int w = 0; w < 4; ++w)
      if (t[w] < best_t[w]) {
        best_t[w] = t[w];
        best[w] = g;
      }
  }
  const double best_ms = best_t[0] + k * best_t[1] + kb * best_t[2] + best_t[3];
  for (size_t c = 0; c < tris_c.size() && st == SEG_OK; ++c) {
    const int g = tris_c[c];
    if (g > s->grid_e_cap) continue;
    s->grid_e = g;
    double t = 0;
    st = time_launches(s, 4, reps, &t);
    if (st == SEG_OK && t < best_e_ms) {
      best_e_ms = t;
      best_e = g;
    }
  }
  // restore the state's data bitwise
  ce = cudaSuccess;
  for (size_t b = 0; b < nkeep && ce == cudaSuccess; ++b)
    ce = cudaMemcpyAsync(keep[b], (char*)saved_x + b * vbytes, vbytes, cudaMemcpyDeviceToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->ctl, saved_ctl, sizeof(DevCtl), cudaMemcpyDeviceToDevice, s->stream);
  for (void* b : {s->Z, s->P0, s->P1, s->Q})
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b, 0, vbytes, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  cudaFree(saved_x);
  cudaFree(saved_ctl);
  if (st == SEG_OK && ce != cudaSuccess) st = fail(SEG_ERR_CUDA, std::string("restore: ") + cudaGetErrorString(ce));
  s->pending = pending;
  for (int w = 0; w < 4; ++w) {
    s->grid[w] = st == SEG_OK ? best[w] : grid0[w];
    out->grid_pass[w] = s->grid[w];
  }
  s->grid_e = st == SEG_OK ? best_e : grid_e0;
  out->grid_blocks = s->grid[kPassCgA];
  out->grid_blocks_energy = s->grid_e;
  out->ms_model = st == SEG_OK ? best_ms : 0.0;
  out->ms_energy = st == SEG_OK ? best_e_ms : 0.0;
  out->cg_weight = k;
  // CG iterations as plain graph nodes before the WHILE node: the iteration
  // count of the latest step (early steps from random data need more)
  if (st == SEG_OK && s->hctl->step > 0) s->cg_peel = std::min(kCgPeelMax, std::max(1, s->hctl->cg_last));
  out->cg_peel = s->cg_peel;
  s->peel_step = s->hctl->step;
  s->peel_it = s->hctl->cg_total;
  // the step graph has the geometry baked in: drop it, the next graph-mode
  // step builds it again
  drop_graph(s);
  return st;
}

seg_status seg_launch_info(seg_state* s, int32_t* grid_blocks, int32_t* block_threads, int32_t* lanes_per_row,
                           int32_t* padded_m) {
  if (!s) return fail(SEG_ERR_ARG, "state is NULL");
  if (grid_blocks) *grid_blocks = s->grid[kPassCgA];
  if (block_threads) *block_threads = kBlockThreads;
  if (lanes_per_row) *lanes_per_row = s->lpr;
  if (padded_m) *padded_m = s->ms;
  return SEG_OK;
}

}  // extern "C"
