"""Python binding of the GB300 eigenfunction-segregation library (libseg.so).

Argument marshalling only: every function forwards to the C entry point of
the same name declared in include/seg.h, and all computation happens in the
library's CUDA kernels.  There is no CPU fallback: importing this package
raises if the compiled library is missing (build it with
``python paper_1408_2355_gb300/build.py``).

Arrays: numpy float64 / int32 / uint8 for host data; torch CUDA tensors are
accepted wherever a device pointer is allowed (``is_device=True``).
"""

from __future__ import annotations

import ctypes as C
import os
import platform

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", platform.machine(), "libseg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libseg.so not found at {LIB_PATH}; build it with `python paper_1408_2355_gb300/build.py`"
    )
lib = C.CDLL(LIB_PATH)

SEG_OK = 0
SEG_ERR_ARG = -1
SEG_ERR_MESH = -2
SEG_ERR_CUDA = -3
SEG_ERR_NO_MEMORY = -4
SEG_ERR_NOT_CONVERGED = -5
SEG_ERR_NONFINITE = -6
SEG_ERR_TIMEOUT = -7
SEG_ERR_UNSUPPORTED = -8

SEG_FP64 = 0
SEG_MIXED_FP32 = 1
SEG_INIT_ONEHOT = 0
SEG_INIT_UNIFORM = 1

EXPORTED = [
    "seg_create_mesh", "seg_mesh_icosphere", "seg_mesh_ellipsoid", "seg_mesh_torus",
    "seg_mesh_dziuk", "seg_mesh_refine", "seg_mesh_info", "seg_mesh_get", "seg_mesh_destroy", "seg_assemble", "seg_assemble_ex", "seg_problem_info",
    "seg_problem_destroy", "seg_state_create", "seg_state_destroy", "seg_set_u", "seg_get_u",
    "seg_step", "seg_step_async", "seg_sync", "seg_substep", "seg_energy",
    "seg_eigenvalue_estimates", "seg_energy_p", "seg_prolong", "seg_continue", "seg_labels", "seg_get_stats",
    "seg_stats_enqueue", "seg_stats_wait", "seg_last_error",
    "seg_time_kernel", "seg_launch_info", "seg_autotune", "seg_s_eps_noalloc",
    "seg_batch_create", "seg_batch_step", "seg_batch_step_async", "seg_batch_sync", "seg_batch_destroy",
    "seg_batch_set_persistent",
    "seg_server_create", "seg_server_submit", "seg_server_tick", "seg_server_info", "seg_server_result",
    "seg_server_clock", "seg_server_destroy", "seg_state_bytes",
    "seg_checkpoint_size", "seg_get_checkpoint", "seg_set_checkpoint", "seg_set_wait_limit", "seg_set_wait_stall",
]


class SegError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"seg status {status}: {message}")
        self.status = status


class seg_params(C.Structure):
    _fields_ = [
        ("cg_rtol", C.c_double),
        ("cg_maxit", C.c_int32),
        ("grid_blocks", C.c_int32),
        ("check_every", C.c_int64),
        ("energy_tol", C.c_double),
        ("launch_mode", C.c_int32),
        ("reserved", C.c_int32),
        ("max_steps", C.c_int64),
        ("wait_limit_ns", C.c_int64),
        ("energy_rtol", C.c_double),
    ]


class seg_stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64),
        ("cg_iterations", C.c_int64),
        ("cg_last", C.c_int32),
        ("cg_max", C.c_int32),
        ("converged", C.c_int32),
        ("status_bits", C.c_int32),
        ("last_check_total", C.c_double),
        ("checks", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("graph_peel", C.c_int32),
        ("reserved", C.c_int32),
    ]


class seg_server_params(C.Structure):
    _fields_ = [
        ("hbm_budget_bytes", C.c_uint64),
        ("max_resident", C.c_int32),
        ("steps_per_tick", C.c_int32),
    ]


SEG_TUNE_MAX = 8


class seg_tune_result(C.Structure):
    _fields_ = [
        ("grid_blocks", C.c_int32),
        ("grid_blocks_energy", C.c_int32),
        ("n_candidates", C.c_int32),
        ("cg_peel", C.c_int32),
        ("cand_grid", C.c_int32 * SEG_TUNE_MAX),
        ("cand_ms", C.c_double * SEG_TUNE_MAX),
        ("ms_model", C.c_double),
        ("ms_energy", C.c_double),
        ("cg_weight", C.c_double),
        ("grid_pass", C.c_int32 * 4),
    ]


class seg_request_info(C.Structure):
    _fields_ = [
        ("phase", C.c_int32),
        ("status", C.c_int32),
        ("steps", C.c_int64),
        ("converged", C.c_int32),
        ("m", C.c_int32),
        ("n_vert", C.c_int64),
        ("total_energy", C.c_double),
        ("t_submit", C.c_double),
        ("t_admit", C.c_double),
        ("t_done", C.c_double),
    ]


_vp = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_d = C.c_double
_pp = C.POINTER(C.c_void_p)

_SIG = {
    "seg_create_mesh": [_vp, _i64, _vp, _i64, _pp],
    "seg_mesh_icosphere": [_i32, _pp],
    "seg_mesh_ellipsoid": [_i32, _d, _d, _d, _pp],
    "seg_mesh_torus": [_i32, _i32, _d, _d, _pp],
    "seg_mesh_dziuk": [_i32, _pp],
    "seg_mesh_refine": [_vp, _vp, _pp, _vp],
    "seg_mesh_info": [_vp, _vp, _vp],
    "seg_mesh_get": [_vp, _vp, _vp],
    "seg_assemble": [_vp, _d, C.c_int, _pp],
    "seg_assemble_ex": [_vp, _d, C.c_int, C.c_uint32, _pp],
    "seg_problem_info": [_vp, _vp, _vp, _vp, _vp],
    "seg_state_create": [_vp, _i32, _d, C.c_int, C.c_uint64, _vp, _vp, _pp],
    "seg_set_u": [_vp, _vp, _i32],
    "seg_get_u": [_vp, _vp, _i32],
    "seg_step": [_vp, _i64, _vp],
    "seg_step_async": [_vp, _i64],
    "seg_sync": [_vp, _vp],
    "seg_substep": [_vp, _i32],
    "seg_energy": [_vp, _vp, _vp, _vp, _vp],
    "seg_eigenvalue_estimates": [_vp, _vp, _vp],
    "seg_energy_p": [_vp, _d, _vp],
    "seg_prolong": [_vp, _vp, _vp],
    "seg_continue": [_vp, _vp, _vp, _d, _d, _vp, _pp, _pp, _pp],
    "seg_labels": [_vp, _vp, _vp],
    "seg_get_stats": [_vp, _vp],
    "seg_stats_enqueue": [_vp, _vp],
    "seg_stats_wait": [_vp, _i32, _vp],
    "seg_time_kernel": [_vp, _i32, _i32, _vp],
    "seg_launch_info": [_vp, _vp, _vp, _vp, _vp],
    "seg_autotune": [_vp, _i32, _vp],
    "seg_s_eps_noalloc": [_vp, _i64, _i32, _vp, _vp, _i64, _d, _vp, _vp],
    "seg_batch_create": [_vp, _i32, _vp, _pp],
    "seg_batch_step": [_vp, _i64],
    "seg_batch_step_async": [_vp, _i64],
    "seg_batch_sync": [_vp],
    "seg_batch_set_persistent": [_vp, _i32],
    "seg_server_create": [_vp, _pp],
    "seg_server_submit": [_vp, _vp, _i32, _d, C.c_int, C.c_uint64, _vp, _vp],
    "seg_server_tick": [_vp, _vp, _vp],
    "seg_server_info": [_vp, _i64, _vp],
    "seg_server_result": [_vp, _i64, _vp],
    "seg_state_bytes": [_vp, _i32, _vp],
    "seg_checkpoint_size": [_vp, _vp],
    "seg_get_checkpoint": [_vp, _vp, C.c_uint64],
    "seg_set_checkpoint": [_vp, _vp, C.c_uint64],
    "seg_set_wait_limit": [_vp, _i64],
    "seg_set_wait_stall": [_vp, _i32],
}
for _name, _args in _SIG.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.seg_server_clock.argtypes = [_vp]
lib.seg_server_clock.restype = C.c_double
for _name in ("seg_mesh_destroy", "seg_problem_destroy", "seg_state_destroy", "seg_batch_destroy",
              "seg_server_destroy"):
    getattr(lib, _name).argtypes = [_vp]
    getattr(lib, _name).restype = None
lib.seg_last_error.argtypes = []
lib.seg_last_error.restype = C.c_char_p


def seg_last_error() -> str:
    return lib.seg_last_error().decode()


def _check(status, ok=(SEG_OK,)):
    if status not in ok:
        raise SegError(status, seg_last_error())
    return status


def _ptr(a):
    """Address of a numpy array or a torch tensor (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(lib, self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh(_Handle):
    _destroy = "seg_mesh_destroy"


class Problem(_Handle):
    _destroy = "seg_problem_destroy"

    def __init__(self, ptr, mesh_keepalive=None):
        super().__init__(ptr)


class State(_Handle):
    _destroy = "seg_state_destroy"

    def __init__(self, ptr, problem, m):
        super().__init__(ptr)
        self.problem = problem  # keep the problem alive while the state exists
        self.m = m


# ------------------------------------------------------------------ meshes


def seg_create_mesh(xyz, tri) -> Mesh:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    out = C.c_void_p()
    _check(lib.seg_create_mesh(_ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], C.byref(out)))
    return Mesh(out)


def seg_mesh_icosphere(level: int) -> Mesh:
    out = C.c_void_p()
    _check(lib.seg_mesh_icosphere(level, C.byref(out)))
    return Mesh(out)


def seg_mesh_ellipsoid(level: int, a: float, b: float, c: float) -> Mesh:
    out = C.c_void_p()
    _check(lib.seg_mesh_ellipsoid(level, a, b, c, C.byref(out)))
    return Mesh(out)


def seg_mesh_torus(nu: int, nv: int, R: float, r: float) -> Mesh:
    out = C.c_void_p()
    _check(lib.seg_mesh_torus(nu, nv, R, r, C.byref(out)))
    return Mesh(out)


SEG_SURFACE_NONE, SEG_SURFACE_ELLIPSOID, SEG_SURFACE_TORUS, SEG_SURFACE_DZIUK = 0, 1, 2, 3


class seg_surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("p0", C.c_double), ("p1", C.c_double),
                ("p2", C.c_double)]


def surface(kind: int, p0: float = 0.0, p1: float = 0.0, p2: float = 0.0) -> seg_surface:
    return seg_surface(kind, 0, p0, p1, p2)


def seg_mesh_dziuk(level: int) -> Mesh:
    out = C.c_void_p()
    _check(lib.seg_mesh_dziuk(level, C.byref(out)))
    return Mesh(out)


def seg_mesh_refine(mesh: Mesh, surf: seg_surface):
    """Returns (fine mesh, parents[n_fine, 2] int32)."""
    n, f = seg_mesh_info(mesh)
    parents = np.empty((n + 3 * f, 2), dtype=np.int32)
    out = C.c_void_p()
    _check(lib.seg_mesh_refine(mesh.ptr, C.byref(surf), C.byref(out), _ptr(parents)))
    fine = Mesh(out)
    return fine, parents[: seg_mesh_info(fine)[0]].copy()


def seg_mesh_info(mesh: Mesh):
    n, f = C.c_int64(), C.c_int64()
    _check(lib.seg_mesh_info(mesh.ptr, C.byref(n), C.byref(f)))
    return n.value, f.value


def seg_mesh_get(mesh: Mesh):
    n, f = seg_mesh_info(mesh)
    xyz = np.empty((n, 3), dtype=np.float64)
    tri = np.empty((f, 3), dtype=np.int32)
    _check(lib.seg_mesh_get(mesh.ptr, _ptr(xyz), _ptr(tri)))
    return xyz, tri


def seg_mesh_destroy(mesh: Mesh):
    mesh.close()


# ---------------------------------------------------------------- assembly


SEG_ASSEMBLE_LUMPED_MASS = 1


def seg_assemble(mesh: Mesh, tau: float, precision: int = SEG_FP64) -> Problem:
    out = C.c_void_p()
    _check(lib.seg_assemble(mesh.ptr, tau, precision, C.byref(out)))
    return Problem(out)


def seg_assemble_ex(mesh: Mesh, tau: float, precision: int = SEG_FP64, flags: int = 0) -> Problem:
    out = C.c_void_p()
    _check(lib.seg_assemble_ex(mesh.ptr, tau, precision, flags, C.byref(out)))
    return Problem(out)


def seg_problem_info(problem: Problem):
    n, nnz, tau, area = C.c_int64(), C.c_int64(), C.c_double(), C.c_double()
    _check(lib.seg_problem_info(problem.ptr, C.byref(n), C.byref(nnz), C.byref(tau), C.byref(area)))
    return {"n_vert": n.value, "nnz": nnz.value, "tau": tau.value, "area": area.value}


def seg_problem_destroy(problem: Problem):
    problem.close()


# ------------------------------------------------------------------- state


def seg_state_create(problem: Problem, m: int, eps: float, init: int = SEG_INIT_UNIFORM, seed: int = 0,
                     params: seg_params | None = None, cuda_stream: int | None = None) -> State:
    out = C.c_void_p()
    pp = C.byref(params) if params is not None else None
    _check(lib.seg_state_create(problem.ptr, m, eps, init, seed & 0xFFFFFFFFFFFFFFFF, pp,
                                C.c_void_p(cuda_stream) if cuda_stream else None, C.byref(out)))
    return State(out, problem, m)


def seg_state_destroy(state: State):
    state.close()


def _n_vert(state: State) -> int:
    return seg_problem_info(state.problem)["n_vert"]


def seg_set_u(state: State, u, is_device: bool = False):
    if not is_device:
        u = np.ascontiguousarray(u, dtype=np.float64)
    _check(lib.seg_set_u(state.ptr, _ptr(u), 1 if is_device else 0))


def seg_get_u(state: State, out=None, is_device: bool = False):
    if out is None:
        out = np.empty((_n_vert(state), state.m), dtype=np.float64)
        is_device = False
    _check(lib.seg_get_u(state.ptr, _ptr(out), 1 if is_device else 0))
    return out


def seg_checkpoint_size(state: State) -> int:
    b = C.c_uint64()
    _check(lib.seg_checkpoint_size(state.ptr, C.byref(b)))
    return b.value


def seg_get_checkpoint(state: State, out=None) -> np.ndarray:
    """The state's checkpoint in a host byte array (see include/seg.h): `out`
    (a contiguous uint8 numpy array of seg_checkpoint_size bytes, e.g. a view
    of pinned memory) or a new one."""
    buf = np.empty(seg_checkpoint_size(state), dtype=np.uint8) if out is None else out
    if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"]:
        raise SegError(SEG_ERR_ARG, "checkpoint buffer must be a contiguous uint8 array")
    _check(lib.seg_get_checkpoint(state.ptr, _ptr(buf), buf.nbytes))
    return buf


def seg_set_checkpoint(state: State, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib.seg_set_checkpoint(state.ptr, _ptr(buf), buf.nbytes))


def seg_set_wait_limit(state: State, ns: int):
    _check(lib.seg_set_wait_limit(state.ptr, int(ns)))


def seg_set_wait_stall(state: State, on: bool):
    _check(lib.seg_set_wait_stall(state.ptr, 1 if on else 0))


def seg_step(state: State, nsteps: int, ok_not_converged: bool = False) -> int:
    done = C.c_int64()
    ok = (SEG_OK, SEG_ERR_NOT_CONVERGED) if ok_not_converged else (SEG_OK,)
    _check(lib.seg_step(state.ptr, nsteps, C.byref(done)), ok)
    return done.value


def seg_step_async(state: State, nsteps: int):
    _check(lib.seg_step_async(state.ptr, nsteps))


def seg_sync(state: State) -> int:
    done = C.c_int64()
    _check(lib.seg_sync(state.ptr, C.byref(done)))
    return done.value


class Batch(_Handle):
    _destroy = "seg_batch_destroy"

    def __init__(self, ptr, states):
        super().__init__(ptr)
        self.states = list(states)  # keep the members alive


def seg_batch_create(states, cuda_stream: int | None = None) -> Batch:
    arr = (C.c_void_p * len(states))(*[s.ptr for s in states])
    out = C.c_void_p()
    _check(lib.seg_batch_create(C.cast(arr, C.c_void_p), len(states),
                                C.c_void_p(cuda_stream) if cuda_stream else None, C.byref(out)))
    return Batch(out, states)


def seg_batch_step(batch: Batch, nsteps: int, ok_not_converged: bool = False):
    ok = (SEG_OK, SEG_ERR_NOT_CONVERGED) if ok_not_converged else (SEG_OK,)
    _check(lib.seg_batch_step(batch.ptr, nsteps), ok)


def seg_batch_step_async(batch: Batch, nsteps: int):
    _check(lib.seg_batch_step_async(batch.ptr, nsteps))


def seg_batch_sync(batch: Batch):
    _check(lib.seg_batch_sync(batch.ptr))


def seg_batch_set_persistent(batch: Batch, on: bool = True):
    _check(lib.seg_batch_set_persistent(batch.ptr, 1 if on else 0))


def seg_batch_destroy(batch: Batch):
    batch.close()


class Server(_Handle):
    _destroy = "seg_server_destroy"

    def __init__(self, ptr):
        super().__init__(ptr)
        self.problems = []  # problems of submitted requests stay alive with the server


def seg_server_create(params: seg_server_params | None = None) -> Server:
    out = C.c_void_p()
    _check(lib.seg_server_create(C.byref(params) if params is not None else None, C.byref(out)))
    return Server(out)


def seg_server_submit(server: Server, problem: Problem, m: int, eps: float, init: int = SEG_INIT_UNIFORM,
                      seed: int = 0, params: seg_params | None = None) -> int:
    rid = C.c_int64()
    _check(lib.seg_server_submit(server.ptr, problem.ptr, m, eps, init, seed & 0xFFFFFFFFFFFFFFFF,
                                 C.byref(params) if params is not None else None, C.byref(rid)))
    server.problems.append(problem)
    return rid.value


def seg_server_tick(server: Server):
    running, queued = C.c_int32(), C.c_int32()
    _check(lib.seg_server_tick(server.ptr, C.byref(running), C.byref(queued)))
    return running.value, queued.value


def seg_server_info(server: Server, rid: int) -> dict:
    info = seg_request_info()
    _check(lib.seg_server_info(server.ptr, rid, C.byref(info)))
    return {k: getattr(info, k) for k, _ in seg_request_info._fields_}


def seg_server_result(server: Server, rid: int):
    info = seg_server_info(server, rid)
    out = np.empty((info["n_vert"], info["m"]), dtype=np.float64)
    _check(lib.seg_server_result(server.ptr, rid, _ptr(out)))
    return out


def seg_server_clock(server: Server) -> float:
    return lib.seg_server_clock(server.ptr)


def seg_server_destroy(server: Server):
    server.close()


def seg_state_bytes(problem: Problem, m: int) -> int:
    b = C.c_uint64()
    _check(lib.seg_state_bytes(problem.ptr, m, C.byref(b)))
    return b.value


def seg_substep(state: State, stage: int):
    _check(lib.seg_substep(state.ptr, stage))


def seg_energy(state: State) -> dict:
    t, f, d, s = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(lib.seg_energy(state.ptr, C.byref(t), C.byref(f), C.byref(d), C.byref(s)))
    return {"total": t.value, "functional": f.value, "dirichlet": d.value, "s_eps": s.value}


def seg_eigenvalue_estimates(state: State):
    lam = np.empty(state.m, dtype=np.float64)
    lam_cl = np.empty(state.m, dtype=np.float64)
    _check(lib.seg_eigenvalue_estimates(state.ptr, _ptr(lam), _ptr(lam_cl)))
    return lam, lam_cl


def seg_energy_p(state: State, p: float) -> float:
    e = C.c_double()
    _check(lib.seg_energy_p(state.ptr, p, C.byref(e)))
    return e.value


def seg_prolong(coarse: State, fine: State, parents):
    parents = np.ascontiguousarray(parents, dtype=np.int32)
    _check(lib.seg_prolong(coarse.ptr, fine.ptr, _ptr(parents)))


def seg_continue(coarse: State, coarse_mesh: Mesh, surf: seg_surface, eps_next: float, tau_next: float,
                 params: seg_params | None = None):
    """Returns (fine mesh, fine problem, fine state)."""
    fm, fp, fs = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(lib.seg_continue(coarse.ptr, coarse_mesh.ptr, C.byref(surf), eps_next, tau_next,
                            C.byref(params) if params is not None else None, C.byref(fm), C.byref(fp),
                            C.byref(fs)))
    mesh = Mesh(fm)
    prob = Problem(fp)
    return mesh, prob, State(fs, prob, coarse.m)


def seg_labels(state: State):
    n = _n_vert(state)
    am = np.empty(n, dtype=np.int32)
    vp = np.empty(n, dtype=np.uint8)
    _check(lib.seg_labels(state.ptr, _ptr(am), _ptr(vp)))
    return am, vp


def seg_get_stats(state: State) -> dict:
    st = seg_stats()
    _check(lib.seg_get_stats(state.ptr, C.byref(st)))
    return {k: getattr(st, k) for k, _ in seg_stats._fields_}


SEG_STATS_RING = 8
SEG_STATS_COPY_BYTES = 3208


def seg_stats_enqueue(state: State) -> int:
    """Ticket for the statistics as of the work enqueued so far (no wait)."""
    t = C.c_int32()
    _check(lib.seg_stats_enqueue(state.ptr, C.byref(t)))
    return t.value


def seg_stats_wait(state: State, ticket: int) -> dict:
    """Wait for the copy behind a ticket only; the statistics it holds."""
    st = seg_stats()
    _check(lib.seg_stats_wait(state.ptr, ticket, C.byref(st)))
    return {k: getattr(st, k) for k, _ in seg_stats._fields_}


def seg_time_kernel(state: State, which: int, reps: int) -> float:
    ms = C.c_double()
    _check(lib.seg_time_kernel(state.ptr, which, reps, C.byref(ms)))
    return ms.value


def seg_launch_info(state: State) -> dict:
    g, b, l, p = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.seg_launch_info(state.ptr, C.byref(g), C.byref(b), C.byref(l), C.byref(p)))
    return {"grid_blocks": g.value, "block_threads": b.value, "lanes_per_row": l.value, "padded_m": p.value}


def seg_autotune(state: State, reps: int = 10) -> dict:
    r = seg_tune_result()
    _check(lib.seg_autotune(state.ptr, reps, C.byref(r)))
    k = r.n_candidates
    return {"grid_blocks": r.grid_blocks, "grid_blocks_energy": r.grid_blocks_energy,
            "candidates": [(r.cand_grid[i], r.cand_ms[i]) for i in range(k)], "ms_model": r.ms_model,
            "ms_energy": r.ms_energy, "cg_weight": r.cg_weight, "cg_peel": r.cg_peel,
            "grid_pass": {"start": r.grid_pass[0], "cg_a": r.grid_pass[1], "cg_b": r.grid_pass[2],
                          "finish": r.grid_pass[3]}}


def _noalloc_args(u, xyz, tri, out):
    """Checks of seg_s_eps_noalloc's arguments, before anything reaches the
    library (which sees only raw device addresses): every array a contiguous
    torch CUDA tensor on the current device with the dtype and shape the C
    entry point reads.  Raises SegError(SEG_ERR_ARG) otherwise."""
    import torch

    def bad(msg):
        raise SegError(SEG_ERR_ARG, "seg_s_eps_noalloc: " + msg)

    named = (("u", u, torch.float64), ("xyz", xyz, torch.float64), ("tri", tri, torch.int32),
             ("out", out, torch.float64))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            bad(f"{name} must be a torch tensor (device memory), not {type(t).__name__}")
        if t.dtype != dt:
            bad(f"{name} must be {dt}, not {t.dtype}")
        if not t.is_contiguous():
            bad(f"{name} must be contiguous")
    if u.ndim != 2:
        bad("u must be (n_vert, m)")
    n_vert, m = int(u.shape[0]), int(u.shape[1])
    if tuple(xyz.shape) != (n_vert, 3):
        bad(f"xyz must be ({n_vert}, 3)")
    if tri.ndim != 2 or tri.shape[1] != 3:
        bad("tri must be (n_tri, 3)")
    if out.numel() < m + 1:
        bad(f"out must hold m + 1 = {m + 1} values")
    for name, t, _ in named:
        if not t.is_cuda:
            bad(f"{name} must be a CUDA tensor")
    dev = torch.cuda.current_device()
    for name, t, _ in named:
        if t.device.index != dev:
            bad(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    return n_vert, m, int(tri.shape[0])


def seg_s_eps_noalloc(u, xyz, tri, eps: float, out, cuda_stream: int | None = None):
    """Allocation-free S_eps and coupling integrals (see include/seg.h).

    u (n_vert x m float64), xyz (n_vert x 3 float64), tri (n_tri x 3 int32)
    and out (m + 1 float64) are caller-owned contiguous CUDA tensors on the
    current device (checked); the call only enqueues work on cuda_stream and
    returns.
    """
    n_vert, m, n_tri = _noalloc_args(u, xyz, tri, out)
    _check(lib.seg_s_eps_noalloc(_ptr(u), n_vert, m, _ptr(xyz), _ptr(tri), n_tri, eps, _ptr(out),
                                 C.c_void_p(cuda_stream) if cuda_stream else None))
