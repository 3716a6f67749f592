/*
 * seg.h -- C ABI of the GB300 eigenfunction-segregation library.
 *
 * The library computes the operator-split gradient flow of Elliott & Ranner,
 * "A computational approach to an optimal partition problem on surfaces"
 * (Algorithm 2.2): m piecewise-linear surface finite-element functions u_i on
 * a triangulated surface Gamma_h are advanced by
 *   step 1  (M + tau K) u~_i = M u_i^k                  (implicit Euler heat step)
 *   step 2  u^_i = u~_i exp(-(2 tau/eps^2) sum_{j!=i} u~_j^2)   (nodal ODE, exact)
 *   step 3  u_i^{k+1} = u^_i / ||u^_i||_{L2(Gamma_h)}   (renormalisation)
 * with M, K the P1 mass and stiffness matrices (Sec. 2.1).  The energies are
 * those of Problem 2.1 and eq. (Seps-u); the eigenvalue estimates are the H^1
 * semi-norms of Sec. 3.2 and the lambda formula of Sec. 1.1.
 *
 * Conventions (all entry points):
 *  - Every call returns a seg_status; SEG_OK == 0.  On error, seg_last_error()
 *    returns a thread-local message.  No call aborts or throws.
 *  - Handles are owned by the library and released with the *_destroy calls.
 *    A seg_problem may be shared read-only by any number of seg_state objects;
 *    it must outlive them.  A seg_mesh may be destroyed after seg_assemble.
 *  - Input arrays are copied.  Output arrays are caller-allocated; unless an
 *    argument says otherwise they are HOST memory and the call returns after
 *    the data is written (it synchronises the state's CUDA stream).
 *  - Vertex-major layout: u[z * m + i] is component i at vertex z, in the
 *    caller's vertex numbering (the library reorders vertices internally for
 *    locality and undoes the permutation on every input and output).
 *  - All device work of a state runs on the CUDA stream given at creation.
 *  - Calls on one state are not thread-safe; distinct states may be used from
 *    distinct threads.
 */
#ifndef SEG_H
#define SEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct seg_mesh seg_mesh;
typedef struct seg_problem seg_problem;
typedef struct seg_state seg_state;

typedef enum {
  SEG_OK = 0,
  SEG_ERR_ARG = -1,            /* invalid argument (null handle, bad size, out-of-range index) */
  SEG_ERR_MESH = -2,           /* degenerate or inconsistent triangulation */
  SEG_ERR_CUDA = -3,           /* a CUDA runtime call failed (message has the CUDA error) */
  SEG_ERR_NO_MEMORY = -4,      /* host or device allocation failed */
  SEG_ERR_NOT_CONVERGED = -5,  /* a step-1 solve reached cg_maxit before cg_rtol */
  SEG_ERR_NONFINITE = -6,      /* a norm or energy became NaN/Inf or a component vanished */
  SEG_ERR_TIMEOUT = -7,        /* a bounded device wait for staged data gave up; the run was halted */
  SEG_ERR_UNSUPPORTED = -8     /* configuration outside the supported range (e.g. m > 32) */
} seg_status;

typedef enum {
  SEG_FP64 = 0,        /* all vectors, matrices and reductions in IEEE float64 */
  SEG_MIXED_FP32 = 1   /* float32 vectors/matrices/exp; inner products, norms, CG
                          alpha/beta and energies accumulated to float64 accuracy */
} seg_precision;

typedef enum {
  SEG_INIT_ONEHOT = 0,  /* Sec. 2.2: one random component set to 1 per vertex */
  SEG_INIT_UNIFORM = 1  /* every component uniform in [0, 1) */
} seg_init;

/* Optional parameters.  Zero-initialise and set what you need; a zero or
 * negative field selects the default given beside it. */
typedef struct {
  double cg_rtol;        /* step-1 CG stops at ||r||_2 <= cg_rtol ||M u||_2 per component;
                            default 1e-12 (SEG_FP64), 1e-7 (SEG_MIXED_FP32).  The solve of
                            step k starts from u^k plus the correction extrapolated from the
                            last solves (y = u~ - u): 3 y_{k-1} - 3 y_{k-2} + y_{k-3} in
                            SEG_MIXED_FP32, 4 y_{k-1} - 6 y_{k-2} + 4 y_{k-3} - y_{k-4} in
                            SEG_FP64, for the components where that prediction beat none in
                            the previous step (none after seg_set_u or creation); its result
                            is the same to this tolerance */
  int32_t cg_maxit;      /* default 1000 */
  int32_t grid_blocks;   /* CUDA blocks of the row kernels (<= 2048); default 2 per SM */
  int64_t check_every;   /* Sec. 2.2 stop rule cadence M_tau; default round(0.1 / tau);
                            the energy check is skipped entirely if set < 0 */
  double energy_tol;     /* stop when |total_k - total_{k - M_tau}| < energy_tol; default
                            1e-6 (Sec. 2.2); a negative value disables stopping */
  int32_t launch_mode;   /* 0 (default): each step is one CUDA graph (built at the first
                            step) whose CG loop runs its first iterations as plain nodes and
                            the rest in a device-controlled WHILE node; 1: the same kernels
                            launched one by one with a host check per CG iteration (slower;
                            for tools that cannot look inside graphs with conditional nodes) */
  int32_t reserved;      /* must be 0 */
  int64_t max_steps;     /* the state stops for good after this many steps (0: no limit); unlike
                            seg_step's nsteps this also holds inside batches and the server */
  int64_t wait_limit_ns; /* limit of each bounded device wait for data staged by the bulk-copy
                            engine (0: 1 s).  A wait that runs out records SEG_ERR_TIMEOUT and
                            halts the run; the copies still in flight are then waited for with
                            the 1 s limit before the kernel returns.  Limits below 2 us are
                            counted in SM clock cycles, 2 per ns */
  double energy_rtol;    /* relative form of the stop rule (0: off): stop also when
                            |total_k - total_{k - M_tau}| <= energy_rtol |total_k|; with
                            check_every = round(dt / tau) it bounds the energy's relative rate of
                            change per simulated time dt, independent of the energy's scale.
                            SEG_ERR_ARG if negative or not finite */
} seg_params;

typedef struct {
  int64_t steps;            /* steps completed since the state was (re)initialised */
  int64_t cg_iterations;    /* total step-1 CG iterations */
  int32_t cg_last;          /* CG iterations of the last completed step */
  int32_t cg_max;           /* largest per-step CG iteration count */
  int32_t converged;        /* 1 once the Sec. 2.2 stop rule fired */
  int32_t status_bits;      /* bit0: a solve hit cg_maxit; bit1: non-finite norm/energy; bit2: timeout */
  double last_check_total;  /* total energy at the latest stop-rule check */
  int64_t checks;           /* number of stop-rule checks evaluated */
  int64_t kernel_launches;  /* hot-path kernel launches on this state (start, CG passes A and B
                               including those that returned at once after the loop ended,
                               finish, energy passes); in a persistent batch, the phases of its
                               launch that ran this state's passes */
  int32_t graph_peel;       /* CG iterations the step graph (launch_mode 0) runs as plain nodes
                               before its loop node (their passes A, and the passes B of all but
                               the last, whose pass B follows the loop condition): the autotuner
                               sets it to the latest step's
                               count; reviews after 3 or more steps (at seg_sync / seg_step, and
                               every 16 steps inside a long seg_step) set it to their mean per
                               step rounded up if that is larger, or smaller by 2 or more (the
                               graph is then rebuilt for the next step) */
  int32_t reserved;         /* 0 */
} seg_stats;

/* ------------------------------------------------------------------ meshes */

/* Sec. 2.1: a triangulated surface Gamma_h.  xyz[n_vert*3] vertex coordinates
 * (float64), tri[n_tri*3] vertex indices (int32, 0-based, outward orientation).
 * Both are copied.  SEG_ERR_ARG for indices out of range or n < 3;
 * SEG_ERR_MESH for a zero-area triangle or a repeated vertex in a triangle. */
seg_status seg_create_mesh(const double* xyz, int64_t n_vert, const int32_t* tri, int64_t n_tri,
                           seg_mesh** out);

/* Unit-sphere icosphere of the given level (N = 10*4^level + 2 vertices, all on
 * |x| = 1): the icosahedron split level times through its edge midpoints. */
seg_status seg_mesh_icosphere(int32_t level, seg_mesh** out);

/* The icosphere mapped radially onto x^2/a^2 + y^2/b^2 + z^2/c^2 = 1. */
seg_status seg_mesh_ellipsoid(int32_t level, double a, double b, double c, seg_mesh** out);

/* Torus ((R + r cos v) cos u, (R + r cos v) sin u, r sin v) on an nu x nv grid,
 * each grid quad split along one fixed diagonal. */
seg_status seg_mesh_torus(int32_t nu, int32_t nv, double R, double r, seg_mesh** out);

/* Surfaces that refinement moves new vertices onto. */
typedef enum {
  SEG_SURFACE_NONE = 0,       /* keep the edge midpoints (the polyhedron itself) */
  SEG_SURFACE_ELLIPSOID = 1,  /* x^2/p0^2 + y^2/p1^2 + z^2/p2^2 = 1 by radial map; p0=p1=p2=1: unit sphere */
  SEG_SURFACE_TORUS = 2,      /* core radius p0, tube radius p1 (p0 > p1 > 0): closest point */
  SEG_SURFACE_DZIUK = 3       /* surface (D) of Sec. 3.4: Phi = (x1 - x3^2)^2 + x2^2 + x3^2 - 1 = 0,
                                 Newton projection x <- x - Phi grad Phi / |grad Phi|^2 until
                                 |Phi| <= 1e-14 (at most 50 iterations) */
} seg_surface_kind;

typedef struct {
  int32_t kind;      /* seg_surface_kind */
  int32_t reserved;  /* must be 0 */
  double p0, p1, p2;
} seg_surface;

/* Surface (D) of Sec. 3.4: the icosahedron's vertices Newton-projected onto
 * Phi = 0, then `level` refinements (seg_mesh_refine with SEG_SURFACE_DZIUK).
 * N = 10*4^level + 2.  SEG_ERR_ARG for level outside [0, 10]. */
seg_status seg_mesh_dziuk(int32_t level, seg_mesh** out);

/* One global refinement (Sec. 3.3 refines the mesh between continuation
 * levels): every triangle is split into four through its edge midpoints and
 * every new vertex is moved onto `surf`.  Numbering: coarse vertices keep
 * their numbers; the midpoint of edge (lo, hi), lo < hi, becomes vertex
 * n_coarse + (rank of the edge in (lo, hi) order); the children of coarse
 * triangle t are t, F + t, 2F + t (at its corners 0, 1, 2) and 3F + t (the
 * middle one).  parents (nullable, host, [n_fine][2] int32) receives the
 * parent edge of every fine vertex ((z, z) for a coarse vertex): the input of
 * seg_prolong.  Refining the level-L icosphere with the unit sphere gives the
 * level-(L+1) icosphere exactly. */
seg_status seg_mesh_refine(const seg_mesh* coarse, const seg_surface* surf, seg_mesh** fine,
                           int32_t* parents);

/* Sizes of a mesh, and a copy of its arrays (either output may be NULL). */
seg_status seg_mesh_info(const seg_mesh* mesh, int64_t* n_vert, int64_t* n_tri);
seg_status seg_mesh_get(const seg_mesh* mesh, double* xyz, int32_t* tri);
void seg_mesh_destroy(seg_mesh* mesh);

/* ---------------------------------------------------------------- assembly */

/* Sec. 2.1 / Algorithm 2.2 step 1: assemble the P1 mass matrix M, stiffness
 * matrix K and A = M + tau K on Gamma_h (float64 on the host, stored on the
 * current CUDA device in the requested precision) for time step tau > 0. */
seg_status seg_assemble(const seg_mesh* mesh, double tau, seg_precision precision,
                        seg_problem** out);

/* seg_assemble with options.  SEG_ASSEMBLE_LUMPED_MASS: the mass-lumped
 * variant -- M is replaced by M_L = diag(row sums of M) = diag(|star(z)|/3)
 * wherever the method uses it (the matrix of step 1, its right-hand side
 * M_L u and the L2 norm of step 3); K, the energies and S_eps are unchanged.
 * SEG_ERR_ARG for an unknown flag. */
#define SEG_ASSEMBLE_LUMPED_MASS 1u
seg_status seg_assemble_ex(const seg_mesh* mesh, double tau, seg_precision precision, uint32_t flags,
                           seg_problem** out);

/* n_vert, number of nonzeros of M/K/A, tau, total area |Gamma_h| (any may be NULL). */
seg_status seg_problem_info(const seg_problem* p, int64_t* n_vert, int64_t* nnz, double* tau,
                            double* area);
void seg_problem_destroy(seg_problem* p);

/* ------------------------------------------------------------------- state */

/* Create the state of m >= 1 components (m <= 32) with penalty eps > 0 and
 * random initial data (Sec. 2.2) drawn on the device from the counter-based
 * generator U(z,i) = (splitmix64(seed ^ splitmix64(z*m+i)) >> 11) * 2^-53,
 * each component then normalised in L2(Gamma_h).  opt may be NULL.
 * cuda_stream is a cudaStream_t (NULL = the library's own stream). */
seg_status seg_state_create(const seg_problem* p, int32_t m, double eps, seg_init init,
                            uint64_t seed, const seg_params* opt, void* cuda_stream,
                            seg_state** out);
void seg_state_destroy(seg_state* s);

/* Replace the state by the L2(Gamma_h)-normalisation of u[n_vert*m] (float64,
 * caller's vertex order).  If is_device != 0, u is a device pointer on the
 * current device, otherwise host memory.  Resets steps, statistics and the
 * stop rule. */
seg_status seg_set_u(seg_state* s, const double* u, int32_t is_device);

/* Write the current normalised state u[n_vert*m] (float64, caller's vertex
 * order) to host memory, or device memory if is_device != 0.  Reading the
 * state (this call, seg_energy, seg_eigenvalue_estimates, seg_labels) does not
 * change the steps that follow. */
seg_status seg_get_u(seg_state* s, double* u, int32_t is_device);

/* Checkpoint and resume (no counterpart in the paper).  A checkpoint holds
 * everything the next step of Algorithm 2.2 reads: the stored state X and its
 * normalisation, the predicted correction of the next solve and the
 * corrections of the last solves it is extrapolated from, the choice of start
 * per component, the stop rule's previous energy and every counter -- in the
 * state's internal vertex order and precision.  seg_set_checkpoint restores it
 * into a state created on the same mesh (the same problem or one assembled
 * from the same mesh, tau and precision) with the same m and eps; the steps
 * that follow are then bitwise those of the run the checkpoint was taken
 * from, provided the restoring state has the same launch geometry
 * (seg_launch_info; the per-block partial sums are added in that order).
 * buf is host memory of seg_checkpoint_size bytes, owned by the caller.
 * seg_get_checkpoint synchronises the state's stream; SEG_ERR_ARG for a
 * buffer too small, a checkpoint of another size, precision, m or eps, or
 * one that is damaged (magic and version are checked). */
seg_status seg_checkpoint_size(seg_state* s, uint64_t* bytes);
seg_status seg_get_checkpoint(seg_state* s, void* buf, uint64_t bytes);
seg_status seg_set_checkpoint(seg_state* s, const void* buf, uint64_t bytes);

/* Change the limit of the bounded device waits of a state (see
 * seg_params.wait_limit_ns; ns <= 0 restores the 1 s default).  Takes effect
 * at the next step; a batch built from the state earlier keeps the limit it
 * was built with. */
seg_status seg_set_wait_limit(seg_state* s, int64_t ns);

/* Testing aid for the failure path (on != 0 / 0 = off).  While on, every
 * staged pass of the state's steps first waits, with the state's wait limit,
 * on a device barrier that nothing completes, so that the wait runs out: the
 * step records SEG_ERR_TIMEOUT and halts the run exactly as when staged data
 * does not arrive in time.  The copies already issued still land and are
 * waited for before the kernel returns; no GPU fault is involved.  Takes
 * effect at the next step (not in batches built earlier). */
seg_status seg_set_wait_stall(seg_state* s, int32_t on);

/* ------------------------------------------------------------------- steps */

/* Algorithm 2.2: advance up to nsteps steps.  Stops early when the Sec. 2.2
 * rule fires (energy change below energy_tol at a check every check_every
 * steps); *steps_done (nullable) receives the steps actually taken.  Returns
 * SEG_ERR_NOT_CONVERGED if any step-1 solve hit cg_maxit (the steps still
 * complete), SEG_ERR_NONFINITE if a norm or energy became non-finite (the run
 * halts).  Synchronises the stream. */
seg_status seg_step(seg_state* s, int64_t nsteps, int64_t* steps_done);

/* As seg_step but only enqueues the work on the state's stream and returns;
 * seg_sync() waits and reports the same status and step count.  (seg_step
 * itself enqueues a run of 64 or more graph-mode steps in chunks of 16, at
 * most two chunks ahead of the device, and adapts the step graph between
 * chunks; seg_step_async enqueues everything at once.) */
seg_status seg_step_async(seg_state* s, int64_t nsteps);
seg_status seg_sync(seg_state* s, int64_t* steps_done);

/* One stage of Algorithm 2.2 on its own (for inspection and testing):
 * stage 1 = heat step (M + tau K) u~ = M u, stage 2 = nodal segregation ODE,
 * stage 3 = L2(Gamma_h) renormalisation.  Stages 1, 2, 3 in order equal one
 * seg_step.  After stage 1 or 2, seg_get_u returns the un-normalised u~ or u^
 * scaled by the current normalisation factors; the state must be brought back
 * with stage 3 (or seg_set_u) before seg_step.  Synchronises. */
seg_status seg_substep(seg_state* s, int32_t stage);

/* --------------------------------------------------------------- batches */

/* Several states advanced together (states of different meshes, m and eps):
 * every pass of a step of Algorithm 2.2 is one kernel launch over all members,
 * and the members' CG loops run inside one device-controlled loop that
 * continues while any member iterates.  Members must share the precision, the
 * lanes-per-row class (padded m: 1-4, 5-8, 9-16 or 17-32 components in
 * float32; 1-2, 3-4, 5-8, 9-16, 17-32 in float64) and the padded matrix row
 * width, and be on one device; n <= 32.  Each member keeps the block
 * decomposition of its own launch geometry (as "virtual" blocks), and a launch
 * of at most the blocks resident at once runs the virtual blocks of every
 * member taking part in the pass, so a member's results are bitwise those of
 * the member stepped alone, and in a CG iteration that only some members need
 * those members have the whole GPU.  The geometry is taken when the batch is
 * built.  While a batch exists its members must not be stepped on their own
 * streams concurrently.
 * cuda_stream = NULL: the batch's own stream. */
typedef struct seg_batch seg_batch;
seg_status seg_batch_create(seg_state* const* states, int32_t n, void* cuda_stream, seg_batch** out);

/* Advance every member by up to nsteps steps (members that meet their stop
 * rule stay where they are); synchronises and returns the first error status
 * of any member (see seg_step).  The _async form only enqueues the work. */
seg_status seg_batch_step(seg_batch* b, int64_t nsteps);
seg_status seg_batch_step_async(seg_batch* b, int64_t nsteps);
seg_status seg_batch_sync(seg_batch* b);
void seg_batch_destroy(seg_batch* b);

/* Persistent mode of a batch (on != 0; 0, the default, restores the step
 * graph).  Each seg_batch_step / seg_batch_step_async call then runs all of
 * its steps of every member in ONE cooperative kernel launch that stays
 * resident on the GPU (one block per SM): every pass of Algorithm 2.2 is a
 * phase over the members' virtual blocks (each member keeps its own block
 * decomposition, so results are bitwise those of the member stepped alone),
 * separated by grid barriers, and the CG loop, the stop rule and the step
 * limits are decided on the device.  The launch ends early once every member
 * has finished.  Barrier waits are bounded (1 s); one that runs out halts
 * every member with SEG_ERR_TIMEOUT.  SEG_ERR_UNSUPPORTED where cooperative
 * launches are not available. */
seg_status seg_batch_set_persistent(seg_batch* b, int32_t on);

/* ----------------------------------------------------------------- serving */

/* A request server with continuous batching: requests (a problem, m, eps,
 * initial data and parameters) are queued; each tick admits queued requests
 * in arrival order while their device footprint fits the memory budget,
 * advances every resident request by steps_per_tick steps -- resident
 * requests of one class (see seg_batch_create) share one batched launch per
 * pass, different classes run on different streams and overlap -- and retires
 * the requests that met their stop rule or step limit (result copied to host
 * memory, device memory released).  A request's result is bitwise the same as
 * when its state is stepped alone.  Problems must outlive their requests.
 * Every request must be able to finish: give it a stop rule (energy_tol >= 0)
 * or max_steps. */
typedef struct seg_server seg_server;

typedef struct {
  uint64_t hbm_budget_bytes;  /* device bytes for resident states; 0: 80% of free memory at creation */
  int32_t max_resident;       /* 0: no limit other than memory */
  int32_t steps_per_tick;     /* 0: 16 */
} seg_server_params;

typedef struct {
  int32_t phase;           /* 0 queued, 1 running, 2 done, 3 failed */
  int32_t status;          /* seg_status (why a request failed) */
  int64_t steps;           /* steps taken */
  int32_t converged;       /* 1: the stop rule fired; 0: the step limit ended it */
  int32_t m;
  int64_t n_vert;
  double total_energy;     /* total energy at the last stop-rule check */
  double t_submit;         /* seconds on the server clock (seg_server_clock) */
  double t_admit;
  double t_done;
} seg_request_info;

seg_status seg_server_create(const seg_server_params* opt, seg_server** out);
/* Queue a request; *id (required) receives its id.  opt as for seg_state_create. */
seg_status seg_server_submit(seg_server* srv, const seg_problem* p, int32_t m, double eps, seg_init init,
                             uint64_t seed, const seg_params* opt, int64_t* id);
/* One scheduling tick (admit, step, retire); running/queued (nullable)
 * receive the counts after the tick.  Synchronises. */
seg_status seg_server_tick(seg_server* srv, int32_t* running, int32_t* queued);
seg_status seg_server_info(seg_server* srv, int64_t id, seg_request_info* out);
/* Final state u[n_vert * m] (float64, caller's vertex order) of a done request. */
seg_status seg_server_result(seg_server* srv, int64_t id, double* u);
/* Seconds since the server was created (host steady clock). */
double seg_server_clock(const seg_server* srv);
void seg_server_destroy(seg_server* srv);

/* Device bytes a state of m components on problem p allocates. */
seg_status seg_state_bytes(const seg_problem* p, int32_t m, uint64_t* bytes);

/* ---------------------------------------------------------------- outputs */

/* Energies of the current state (Problem 2.1, eq. (Seps-u), tables of Sec. 3):
 *   total      = sum_i D_i + S_eps   (the paper's reported "total energy")
 *   functional = 0.5 sum_i D_i + S_eps   (E^{eps,h})
 *   dirichlet  = sum_i D_i, D_i = int |grad u_i|^2 = u_i^T K u_i
 *   s_eps      = eps^-2 int sum_i sum_{j!=i} u_i^2 u_j^2 (exact quadrature)
 * Any output pointer may be NULL. */
seg_status seg_energy(seg_state* s, double* total, double* functional, double* dirichlet,
                      double* s_eps);

/* Eigenvalue estimates per component (host arrays of length m, nullable):
 * lambda[i] = D_i (Sec. 3.2: the H^1 semi-norm of the normalised component),
 * lambda_cl[i] = D_i + (2/eps^2) int u_i^2 sum_{j!=i} u_j^2 (the formula of Sec. 1.1). */
seg_status seg_eigenvalue_estimates(seg_state* s, double* lambda, double* lambda_cl);

/* The l^p energy of Problem 1.2 from the eigenvalue estimates lambda[i] = D_i:
 * ((1/m) sum_i lambda_i^p)^(1/p) for 1 <= p < inf, max_i lambda_i for
 * p = +inf (pass INFINITY).  SEG_ERR_ARG for p < 1 or NaN. */
seg_status seg_energy_p(seg_state* s, double p, double* e_p);

/* Start `fine` from the P1 interpolation of `coarse`'s current state on a
 * refined mesh (Sec. 3.3: the previous level's minimiser is the initial
 * condition of the next): u_fine(z) = (u(parents[2z]) + u(parents[2z+1]))/2,
 * parents as written by seg_mesh_refine (host array, [n_fine][2], copied).
 * The result replaces fine's state like seg_set_u (normalised in fine's L2
 * norm before its next step).  Both states need the same m; all arithmetic
 * runs on the device.  SEG_ERR_ARG for mismatched sizes or a parent index
 * out of range. */
seg_status seg_prolong(seg_state* coarse, seg_state* fine, const int32_t* parents);

/* One level of the continuation of Sec. 3.3: refine coarse_mesh onto `surf`
 * (seg_mesh_refine), assemble with tau_next in coarse's precision and
 * assembly flags, create a state with eps_next and `opt` (NULL: defaults) on
 * a new stream, and start it from the P1 interpolation of coarse
 * (seg_prolong).  The caller owns the three outputs.  The paper's rule
 * divides eps and tau by sqrt(2) per bisection level; one refinement here
 * equals two bisection levels, so eps_next = eps / 2, tau_next = tau / 2. */
seg_status seg_continue(seg_state* coarse, const seg_mesh* coarse_mesh, const seg_surface* surf,
                        double eps_next, double tau_next, const seg_params* opt, seg_mesh** fine_mesh,
                        seg_problem** fine_problem, seg_state** fine_state);

/* Partition read-out per vertex (host arrays of length n_vert, nullable):
 * argmax[z] = argmax_i u_i(z) (lowest index on ties); v_positive[z] = 1 if
 * v_i(z) = u_i(z) - sum_{j!=i} u_j(z) > 0 for that i (eq. (vi)), else 0. */
seg_status seg_labels(seg_state* s, int32_t* argmax, uint8_t* v_positive);

/* Statistics of the state (synchronises its stream). */
seg_status seg_get_stats(seg_state* s, seg_stats* out);

/* Statistics without waiting for later work: seg_stats_enqueue enqueues on
 * the state's stream a copy of the statistics as they will be once the work
 * enqueued so far is done (into one of SEG_STATS_RING pinned slots) and
 * returns a ticket (>= 0); seg_stats_wait waits for that copy only -- not
 * for steps enqueued after it -- and fills *out as seg_get_stats would then
 * have.  A loop that enqueues step k + 1 before it waits for step k's
 * statistics reads every step's result while the device keeps stepping.  A
 * ticket stays valid until SEG_STATS_RING more copies have been enqueued
 * (SEG_ERR_ARG after that, or for a ticket never issued).  Each copy moves
 * SEG_STATS_COPY_BYTES bytes (the state's control block) from the device. */
#define SEG_STATS_COPY_BYTES 3208
#define SEG_STATS_RING 8
seg_status seg_stats_enqueue(seg_state* s, int32_t* ticket);
seg_status seg_stats_wait(seg_state* s, int32_t ticket, seg_stats* out);

/* Thread-local description of the last error of this thread ("" if none). */
const char* seg_last_error(void);

/* -------------------------------------------------------------- diagnostics */

/* Time `reps` back-to-back launches of one hot-path kernel of this state on
 * its stream with CUDA events; *ms_per_launch receives the mean.  which:
 * 0 = start pass (residual, norms, Dirichlet energy), 1 = CG pass A (A p +
 * p.Ap) as in the first iteration of a solve (p = z, the only form a solve of
 * one iteration runs), 8 = CG pass A as in a later even iteration (also the
 * direction update p = z + beta p), 6 = CG pass A as in an odd iteration
 * (which also applies the two pending solution updates), 2 = CG pass B
 * (residual update + dots) in a later iteration, 9 = CG pass B in the first
 * iteration of a solve that goes on (which also copies p_1 = z_0 out of the
 * residual buffer), 3 = finish pass (last solution update + nodal ODE)
 * with one pending update, 7 = the same with two (after an odd count of 3 or
 * more), 4 = energy pass of the stop rule (S_eps), 5 = energy pass with the
 * per-component coupling integrals.  The kernels run on the state's own
 * buffers, so the state's values are undefined afterwards: call seg_set_u
 * (or seg_set_checkpoint) before using it. */
seg_status seg_time_kernel(seg_state* s, int32_t which, int32_t reps, double* ms_per_launch);

/* Launch geometry of the row kernels of a state (nullable outputs);
 * grid_blocks is the grid of CG pass A (the autotuner may give each pass its
 * own). */
seg_status seg_launch_info(seg_state* s, int32_t* grid_blocks, int32_t* block_threads,
                           int32_t* lanes_per_row, int32_t* padded_m);

/* ---------------------------------------------------------------- autotuner */

#define SEG_TUNE_MAX 8
typedef struct {
  int32_t grid_blocks;         /* chosen blocks of the row kernels */
  int32_t grid_blocks_energy;  /* chosen blocks of the energy-check kernel */
  int32_t n_candidates;        /* row grids tried (first SEG_TUNE_MAX listed) */
  int32_t cg_peel;             /* CG iterations the step graph now runs before its loop node */
  int32_t cand_grid[SEG_TUNE_MAX];
  double cand_ms[SEG_TUNE_MAX]; /* modelled step time of each row grid, ms */
  double ms_model;             /* modelled step time of the chosen row grid */
  double ms_energy;            /* one energy check with the chosen grid, ms */
  double cg_weight;            /* CG iterations per step used in the model */
  int32_t grid_pass[4];        /* chosen blocks of the start pass, CG pass A, CG pass B, finish */
} seg_tune_result;

/* Pick the launch geometry of a state by measurement (no counterpart in the
 * paper; the arithmetic of Algorithm 2.2 is unchanged).  The row grid (and
 * with it the block of rows each CUDA block owns) is chosen among 1 or 2
 * blocks per SM and 2 or 4 waves of 2 blocks per SM (at most one block per
 * 256 rows, at most 2048 blocks), separately for each of the four row
 * passes (start, CG pass A, CG pass B, finish): each pass keeps the candidate
 * with its shortest time, the mean of `reps` (<= 0: 10) timed launches.
 * cand_ms[c] is the modelled step time t_start + k (t_cgA + t_cgB) + t_finish
 * with all passes on candidate c, ms_model the same with each pass on its
 * chosen grid, k the state's CG iterations per step so far (8 before its
 * first step); grid_blocks is CG pass A's grid.  The energy-check grid
 * among 1 or 2 blocks per SM and 2 or 4 waves of 2 blocks per SM by its own
 * time.  The state's data and
 * counters are saved before and restored bitwise after the timing launches,
 * and its step graph is rebuilt with the chosen geometry and with cg_peel =
 * the CG iterations of the state's latest step (1 .. 16; unchanged before
 * the first step) as plain graph nodes ahead of the
 * conditional loop node (passes after convergence return at once; an
 * evaluation of the loop condition costs more); later syncs review the peel
 * (seg_stats.graph_peel).  Later steps give
 * the same results as without tuning up to the summation order of the
 * per-block partial inner products.  A batch built from the state earlier
 * keeps the geometry it was built with.  Needs device memory for four (five
 * in SEG_FP64) state-sized vectors (the state, the predicted correction and
 * the corrections of the last solves; SEG_ERR_NO_MEMORY otherwise).
 * Synchronises. */
seg_status seg_autotune(seg_state* s, int32_t reps, seg_tune_result* out);

/* ------------------------------------------------------- allocation-free call */

/* The paper has no counterpart of this entry point.  It is for callers that
 * cannot allocate device memory -- a process whose GPU memory is reserved up
 * front by another framework's allocator, code running while a CUDA graph is
 * captured (allocation is not allowed then), or a loop whose latency budget an
 * allocation would break.  It computes, from caller-owned DEVICE buffers on the
 * current device,
 *   out[0]     = S_eps = eps^-2 sum_i c_i
 *   out[1 + i] = c_i   = int_{Gamma_h} u_i^2 sum_{j != i} u_j^2   (i < m)
 * for u[n_vert * m] (float64, vertex-major, caller's numbering, normalised as
 * the caller wishes), xyz[n_vert * 3] (float64) and tri[n_tri * 3] (int32; a
 * triangle with an index outside [0, n_vert) contributes nothing).  out holds
 * m + 1 float64 values.  The work is enqueued on cuda_stream (NULL = the legacy
 * default stream) and the call returns without waiting.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (per-block partial sums and a completion counter) is a fixed 64 KiB device
 * array inside the library, which every GPU that loads the library keeps until
 * the process exits.  Limit: m <= 32 (SEG_ERR_UNSUPPORTED otherwise).
 * The first call on a device looks up the address of that array
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  All calls on a device share the array: calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Each call clears the completion counter first. */
seg_status seg_s_eps_noalloc(const double* u, int64_t n_vert, int32_t m, const double* xyz,
                             const int32_t* tri, int64_t n_tri, double eps, double* out,
                             void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SEG_H */
