// Internal definitions shared by the host orchestration and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "seg.h"

namespace segimpl {

constexpr int kMaxCols = 32;       // padded components per vertex row
constexpr int kBlockThreads = 384;  // threads per block of every row kernel
constexpr int kMaxDots = 6;         // inner products fused into one pass
// Resident blocks per SM the row passes are compiled for (register bound)
// and launched with; the triangle passes use kTriBlocksPerSM.
constexpr int kRowBlocksPerSM = 2;
constexpr int kTriBlocksPerSM = 2;
constexpr int kStartBlocksPerSM = 1;  // the start pass (more registers per thread)
constexpr int kMaxGrid = 2048;  // blocks of one kernel of a state
constexpr int kTuneWaves = 4;   // the autotuner tries up to this many waves of blocks
constexpr int kCgUnroll = 2;    // CG iterations per evaluation of the step graph's loop condition
constexpr int kCgPeelDefault = 4;  // CG iterations placed before the loop (the autotuner adjusts it)
constexpr int kCgPeelMax = 16;
constexpr int kNumCounters = 8;    // last-block tickets, one per kernel kind
constexpr unsigned long long kDefaultWaitNs = 1000000000ull;  // bounded waits for staged data: 1 s

enum RowPass { kPassStart = 0, kPassCgA = 1, kPassCgB = 2, kPassFinish = 3 };
enum CounterSlot { kCtrStart = 0, kCtrCgA = 1, kCtrCgB = 2, kCtrEnergy = 3, kCtrFinish = 4 };

// Device-resident control block: per-component scalars of the solve and the
// step loop.  Written only by the last block of a reduction kernel (or by one
// thread), read by the following kernels; the host copies it back at sync
// points.
struct DevCtl {
  double n2[kMaxCols];        // ||X_i||_M^2 of the stored (un-normalised) components
  double inv_n[kMaxCols];     // scale of the represented state u_i = X_i * inv_n[i]
  double lam[kMaxCols];       // D_i = u_i^T K u_i of the normalised state
  double tol2[kMaxCols];      // (cg_rtol ||M X_i||_2)^2
  double rz[kMaxCols];        // r^T D^-1 r of the current CG iterate
  double rr0[kMaxCols];       // ||r_0||_2^2, the initial residual of the current solve
  double alpha[2][kMaxCols];  // CG step length of the last two iterations
  double beta[kMaxCols];      // CG direction update factor
  double coup[kMaxCols];      // int u_i^2 sum_{j != i} u_j^2 (normalised state)
  int active[kMaxCols];       // component still iterating in the current solve
  int carry[kMaxCols];        // the next solve starts from the predicted correction in Y (else from y = 0)
  double ysc[kMaxCols];       // scale (1 or 0) of the predicted correction in the current solve
  int it;                     // CG iterations completed in the current solve
  int cont;                   // loop-continue flag (mirrors the graph conditional)
  int halted;                 // 0 running, 1 stop rule met, 2 error
  int status;                 // bit0: solve hit maxit, bit1: non-finite value, bit2: timeout
  long long step;             // steps completed
  long long cg_total;         // total CG iterations
  int cg_last;
  int cg_max;
  long long checks;           // stop-rule checks evaluated
  double e_total;             // last energy evaluation: sum D + S_eps
  double e_dir;
  double e_s;
  double e_prev;              // total of the previous stop-rule check
  int have_prev;
  int dir_in_z;               // the solve ended after one iteration in CG pass A: its direction p_1 = z_0 is in Z
  long long step_mark;        // ctl->step when the last batch of steps was enqueued
  unsigned long long launches;  // hot-path kernel launches (block 0 counts each)
  unsigned int counters[kNumCounters];
};
// seg_stats_enqueue copies the whole control block.
static_assert(sizeof(DevCtl) == SEG_STATS_COPY_BYTES, "size of the control block");

// Arguments of every hot-path kernel (passed by value; identical struct for
// all kernels of a state so that one graph node layout fits all).
template <typename T>
struct KArgs {
  int n;    // vertex rows
  int m;    // components
  int ms;   // padded components (row stride)
  int ell_w;       // entries per padded-ELL row (8 or 16)
  const int* ell_col;  // [n][ell_w] column indices; padding repeats the row itself
  const T* valA;   // [n][ell_w] A = M + tau K (0 on padding)
  const T* valM;
  const T* valK;
  const T* dinv;   // 1 / diag(A)
  const T* diagA;  // diag(A)
  T* X;            // state (the step's right-hand side is M X)
  T* Y;            // CG iterate x = X + y; y starts at a prediction of the step's correction
  T* H0;           // the corrections y of the last two (float) or three (double)
  T* H1;           // solves, step k's in H[k % 2] or H[k % 3]
  T* H2;           // (double only)
  T* Z;            // preconditioned residual z = D^-1 r
  T* P0;           // search directions (ping-pong between CG iterations)
  T* P1;
  T* Q;            // A p
  DevCtl* ctl;
  void* part;      // per-block partial sums
  double tau;
  double coef;     // 2 tau / eps^2
  double inv_eps2;
  double rtol2;
  int maxit;
  int set_cond;    // 1 when launched inside the step graph
  unsigned long long cond;  // cudaGraphConditionalHandle of the CG loop
  // energy pass
  const int* tri;  // [F][3] rows of the triangle corners (internal numbering)
  const T* tarea;  // |T|
  int ntri;
  long long check_every;
  double energy_tol;
  double energy_rtol;  // relative form of the stop rule (0: off)
  int force;       // timing/forced launches: energy regardless of the cadence, CG passes regardless of the loop state
  int apply_x;     // finish pass: x = X + y with the lagged CG updates of y (else x = X)
  int apply_ode;   // finish pass: apply the nodal segregation ODE
  int count_step;  // finish pass: increment the step counter
  int ignore_halt; // run even if the control block is halted (direct calls)
  long long max_steps;  // > 0: the state is finished once step >= max_steps
  unsigned long long wait_ns;  // limit of one bounded wait for staged data (default 1 s)
  int stall_waits;             // testing aid: the staged passes first wait on a barrier nothing completes
  int norm_only;   // start pass: the normalisation and D_i only (reading the state between steps)
};

// True if a step pass must not touch this state: it halted (stop rule or
// error) or reached its step limit.  Every block reads the same values, so
// the decision is uniform over the grid.
template <typename T>
__device__ __forceinline__ bool state_finished(const KArgs<T>& a, const DevCtl* ctl) {
  if (a.ignore_halt) return false;
  return ctl->halted != 0 || (a.max_steps > 0 && ctl->step >= a.max_steps);
}

// Arguments of a batched launch.  Member i keeps the block decomposition it
// has when stepped alone: vg[i] virtual blocks, each running the member's
// pass body with the arguments tab[i] exactly as block vb of its own grid
// would.  The launch has a fixed grid of physical blocks (as many as are
// resident at once) that take the virtual blocks of the members taking part
// in the pass in turn, so results are bitwise those of each member alone and
// a member that has stopped iterating leaves the whole GPU to the others.
constexpr int kMaxBatch = 32;
enum BatchMap { kMapAll = 0, kMapCgA = 1, kMapCgB = 2 };
template <typename T>
struct BatchArgs {
  KArgs<T> tab[kMaxBatch];  // in the kernel's parameter space (read through the constant cache)
  int ninst;
  int vg[kMaxBatch];        // virtual blocks (own grid) of each member in this pass
  int map;                  // BatchMap: which members take part
  int* amap;                // [kMaxBatch] members iterating in the current CG iteration (device)
  unsigned long long cond;  // conditional handle of the batch's CG loop
};

// A persistent batched launch runs whole steps of every member in one
// cooperative kernel: each pass of Algorithm 2.2 is a phase in which the
// physical blocks take the members' virtual blocks (as in BatchArgs), and a
// grid barrier separates the phases.  The block that arrives last at a
// barrier publishes what the next phase needs (which members take part, and
// whether the CG loop goes on), so that every block reads the same values.
struct PersistCtl {
  unsigned int count;   // blocks arrived at the current barrier
  unsigned int gen;     // barrier generation (released by the last arrival)
  int status;           // bit 0: a barrier wait ran out
  int go;               // the CG loop runs another pass B
  int active;           // some member still steps
  int pad;
  int map_a[kMaxBatch];  // members of the next CG pass A
  int map_b[kMaxBatch];  // members of the next CG pass B
};
constexpr int kNumPhasePasses = 5;  // start, CG pass A, CG pass B, finish (RowPass order), then the energy check
template <typename T>
struct PersistArgs {
  KArgs<T> tab[kMaxBatch];  // in the kernel's parameter space
  int ninst;
  int vg[kNumPhasePasses][kMaxBatch];  // virtual blocks of each member in each pass (its own grids)
  PersistCtl* pc;
  long long nsteps;
  unsigned long long wait_ns;  // limit of one barrier wait
};
// (kernel parameters: at most 32 764 bytes per launch)
static_assert(sizeof(PersistArgs<double>) <= 32764 && sizeof(BatchArgs<double>) <= 32764,
              "batched arguments exceed the kernel parameter space");

// Function table of one (precision, lanes-per-row) specialisation.
struct KernelSet {
  void* start;
  void* cg_a;
  void* cg_b;
  void* finish;
  void* energy;        // S_eps and per-component coupling integrals
  void* energy_check; // S_eps only (stop rule, seg_energy)
  void* init_rng;     // (args, perm, seed, kind)
  void* scatter_in;   // (args, src, perm)
  void* gather_out;   // (args, dst, iperm)
  void* labels;       // (args, am, vp, iperm)
  void* b_start;        // batched passes (BatchArgs)
  void* b_cg_a;
  void* b_cg_b;
  void* b_finish;
  void* b_energy_check;
  void* b_vote;         // one block: the batch's CG loop condition
  void* persist;        // persistent batched steps (PersistArgs, cooperative launch)
  unsigned smem_start;  // dynamic shared memory of k_start (bytes)
  unsigned smem_cg_a;   // dynamic shared memory of k_cg_a (bytes)
};

bool get_kernels_f32(int lpr, int ell_w, KernelSet* ks);
bool get_kernels_f64(int lpr, int ell_w, KernelSet* ks);

// Record the message returned by seg_last_error() on this thread.
void set_last_error(const char* msg);
const char* last_error();

// Key equal for states that may share a batch (precision, lanes per row,
// padded matrix row width, device).
long long state_class_key(const seg_state* s);

// Host-side mesh and assembly (mesh.cpp / assemble.cpp).
struct HostMesh {
  std::vector<double> xyz;  // [n][3]
  std::vector<int32_t> tri;  // [f][3]
  int64_t n = 0, f = 0;
};

std::string validate_mesh(const HostMesh& m, seg_status* code);
void make_icosphere(int level, HostMesh* out);
void make_dziuk(int level, HostMesh* out);
void make_torus(int nu, int nv, double R, double r, HostMesh* out);

// Surface that refinement projects new vertices onto (seg_surface of seg.h).
struct SurfaceDesc {
  int kind;
  double p0, p1, p2;
};
void project_point(double* p, const SurfaceDesc& s);
void refine_mesh(const HostMesh& in, const SurfaceDesc& surf, HostMesh* out, std::vector<int32_t>* parents);

struct HostCSR {
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> M, K;
  std::vector<double> area;   // per triangle (internal order = input order)
  std::vector<int32_t> perm;   // internal row -> caller vertex
  std::vector<int32_t> iperm;  // caller vertex -> internal row
  std::vector<int32_t> tri_rows;  // triangles in internal row numbering
};

void assemble_p1(const HostMesh& mesh, HostCSR* out);

}  // namespace segimpl
