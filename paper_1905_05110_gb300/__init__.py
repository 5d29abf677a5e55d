"""GB300-native volume-penalization lattice Boltzmann (VP-LBM) for rigid-body FSI.

Thin Python binding of the C ABI declared in ``include/vplbm.h``.  Every
function named ``vplbm_*`` here marshals its arguments and calls the entry
point of the same name in ``libvplbm.so``; all of the time stepping runs in
the library's CUDA kernels.  PyTorch is used only for device memory (the
``Simulation`` class allocates the library's buffers as torch tensors) and for
the CUDA stream handle.

If the library has not been built, or no CUDA device is present, the calls
raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "VplbmError", "load_library", "lattice_desc", "body_desc", "Simulation",
    "vplbm_create", "vplbm_create_with_buffers", "vplbm_buffer_sizes_for", "vplbm_destroy",
    "vplbm_init_equilibrium", "vplbm_set_populations", "vplbm_step", "vplbm_sync",
    "vplbm_get_populations", "vplbm_get_fields", "vplbm_get_fields_dev", "vplbm_get_history",
    "vplbm_get_body", "vplbm_create_bodies", "vplbm_get_num_bodies", "vplbm_get_history_body",
    "vplbm_get_body_k", "MAX_BODIES", "vplbm_set_launch", "vplbm_get_launch", "vplbm_autotune",
    "vplbm_get_launch_count", "vplbm_get_kernel_launches", "vplbm_eval_recip_f32", "LAUNCH_KINDS", "vplbm_save", "vplbm_load", "vplbm_last_error", "vplbm_version",
    "vplbm_step_noalloc", "BodyState", "vplbm_inject_wait_timeout", "Batch",
    "vplbm_batch_create", "vplbm_batch_destroy", "vplbm_batch_member", "vplbm_batch_step",
    "vplbm_batch_sync", "vplbm_batch_set_launch", "vplbm_batch_get_launch", "vplbm_batch_autotune",
    "vplbm_batch_set_mode", "vplbm_batch_get_mode", "vplbm_batch_set_persistent",
    "vplbm_batch_get_persistent", "vplbm_batch_inject_barrier_timeout",
    "EXPORTED_SYMBOLS", "RECORD_FIELDS",
]

Q = 9
STATUS = {0: "VPLBM_OK", 1: "VPLBM_EINVAL", 2: "VPLBM_ENOMEM", 3: "VPLBM_ECUDA",
          4: "VPLBM_ENONFINITE", 5: "VPLBM_ETIMEOUT", 6: "VPLBM_EUNSUPPORTED",
          7: "VPLBM_ERANGE", 8: "VPLBM_EIO"}
PRECISIONS = {"f64": 0, "f32": 1, "f16": 2}
BC_KINDS = {"periodic": 0, "noslip": 1, "velocity": 2, "zerograd": 3, "symmetry": 4, "convective": 5}
MOTIONS = {"fixed": 0, "imposed": 1, "free": 2}
SIDES = ("west", "east", "south", "north")
RECORD_FIELDS = ("t", "fx", "fy", "torque", "cd", "cl", "x", "y", "theta",
                 "vx", "vy", "omega", "fpen_x", "fpen_y", "tpen", "n_solid")


class VplbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


# ---- C structs (mirrors of include/vplbm.h) ----------------------------------

class BC(C.Structure):
    _fields_ = [("kind", C.c_int), ("ux", C.c_double), ("uy", C.c_double),
                ("ux_profile", C.POINTER(C.c_double)), ("uy_profile", C.POINTER(C.c_double))]


class LatticeDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("s", C.c_double * 9), ("eta", C.c_double),
                ("rho0", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
                ("bc", BC * 4), ("precision", C.c_int), ("collision", C.c_int)]


class BodyDesc(C.Structure):
    _fields_ = [("radius", C.c_double), ("x", C.c_double), ("y", C.c_double),
                ("theta", C.c_double), ("vx", C.c_double), ("vy", C.c_double),
                ("omega", C.c_double), ("motion", C.c_int), ("axis", C.c_int),
                ("amp", C.c_double), ("freq", C.c_double), ("phase", C.c_double),
                ("mass", C.c_double), ("inertia", C.c_double),
                ("damp", C.c_double * 3), ("stiff", C.c_double * 3),
                ("q0", C.c_double * 3), ("f_ext", C.c_double * 3),
                ("dof_mask", C.c_uint), ("u_ref", C.c_double), ("d_ref", C.c_double),
                ("shape", C.c_int), ("radius_b", C.c_double)]


class Record(C.Structure):
    _fields_ = [(n, C.c_double) for n in RECORD_FIELDS]


class BufferSizes(C.Structure):
    _fields_ = [(n, C.c_size_t) for n in
                ("populations", "body_state", "partials", "history", "profiles", "control")]


class Buffers(C.Structure):
    _fields_ = [("populations_dev", C.c_void_p * 2), ("body_state_dev", C.c_void_p),
                ("partials_dev", C.c_void_p), ("history_dev", C.c_void_p),
                ("profiles_dev", C.c_void_p), ("control_dev", C.c_void_p)]


class AdjointDesc(C.Structure):
    _fields_ = [("nsteps", C.c_longlong), ("window_start", C.c_longlong), ("w_cd", C.c_double),
                ("w_cl", C.c_double), ("checkpoint_interval", C.c_longlong)]


class BodyState(C.Structure):
    _fields_ = [("q", C.c_double * 3), ("v", C.c_double * 3), ("step", C.c_longlong),
                ("error", C.c_int), ("pad", C.c_int)]


_D = C.POINTER(C.c_double)
_CTX = C.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "vplbm_buffer_sizes_for": (C.c_int, [C.POINTER(LatticeDesc), C.POINTER(BodyDesc), C.c_longlong,
                                         C.POINTER(BufferSizes)]),
    "vplbm_create": (C.c_int, [C.POINTER(LatticeDesc), C.POINTER(BodyDesc), C.c_longlong, C.c_void_p,
                               C.POINTER(_CTX)]),
    "vplbm_create_with_buffers": (C.c_int, [C.POINTER(LatticeDesc), C.POINTER(BodyDesc), C.c_longlong,
                                            C.c_void_p, C.POINTER(Buffers), C.POINTER(_CTX)]),
    "vplbm_destroy": (None, [_CTX]),
    "vplbm_init_equilibrium": (C.c_int, [_CTX, _D, _D, _D]),
    "vplbm_set_populations": (C.c_int, [_CTX, _D]),
    "vplbm_step": (C.c_int, [_CTX, C.c_longlong]),
    "vplbm_sync": (C.c_int, [_CTX]),
    "vplbm_get_populations": (C.c_int, [_CTX, _D]),
    "vplbm_get_fields": (C.c_int, [_CTX, _D, _D, _D]),
    "vplbm_get_fields_dev": (C.c_int, [_CTX, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vplbm_get_history": (C.c_int, [_CTX, C.c_longlong, C.c_longlong, C.POINTER(Record)]),
    "vplbm_get_body": (C.c_int, [_CTX, _D, _D, C.POINTER(C.c_longlong)]),
    "vplbm_create_bodies": (C.c_int, [C.POINTER(LatticeDesc), C.POINTER(BodyDesc), C.c_int, C.c_longlong,
                                      C.c_void_p, C.POINTER(_CTX)]),
    "vplbm_get_num_bodies": (C.c_int, [_CTX, C.POINTER(C.c_int)]),
    "vplbm_get_history_body": (C.c_int, [_CTX, C.c_int, C.c_longlong, C.c_longlong, C.POINTER(Record)]),
    "vplbm_get_body_k": (C.c_int, [_CTX, C.c_int, _D, _D, C.POINTER(C.c_longlong)]),
    "vplbm_set_launch": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_int]),
    "vplbm_get_launch": (C.c_int, [_CTX, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "vplbm_autotune": (C.c_int, [_CTX, C.c_int]),
    "vplbm_get_launch_count": (C.c_int, [_CTX, C.POINTER(C.c_longlong)]),
    "vplbm_get_kernel_launches": (C.c_int, [_CTX, C.POINTER(C.c_longlong)]),
    "vplbm_eval_recip_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "vplbm_inject_wait_timeout": (C.c_int, [_CTX, C.c_int]),
    "vplbm_save": (C.c_int, [_CTX, C.c_char_p]),
    "vplbm_load": (C.c_int, [_CTX, C.c_char_p]),
    "vplbm_step_noalloc": (C.c_int, [C.POINTER(LatticeDesc), C.POINTER(BodyDesc), C.c_void_p * 2,
                                     C.c_void_p, C.c_void_p, C.c_longlong, C.c_longlong, C.c_void_p]),
    "vplbm_batch_create": (C.c_int, [C.POINTER(LatticeDesc), C.c_void_p, C.c_int, C.c_longlong, C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "vplbm_batch_destroy": (None, [C.c_void_p]),
    "vplbm_batch_member": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(_CTX)]),
    "vplbm_batch_step": (C.c_int, [C.c_void_p, C.c_longlong]),
    "vplbm_batch_sync": (C.c_int, [C.c_void_p]),
    "vplbm_batch_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "vplbm_batch_get_launch": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "vplbm_batch_autotune": (C.c_int, [C.c_void_p, C.c_int]),
    "vplbm_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "vplbm_batch_get_mode": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "vplbm_batch_set_persistent": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    "vplbm_batch_get_persistent": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int)] * 5 + [C.POINTER(C.c_longlong)]),
    "vplbm_batch_inject_barrier_timeout": (C.c_int, [C.c_void_p, C.c_int]),
    "vplbm_adjoint": (C.c_int, [_CTX, C.c_void_p, _D, _D]),
    "vplbm_last_error": (C.c_char_p, []),
    "vplbm_version": (C.c_char_p, []),
}
EXPORTED_SYMBOLS = tuple(_SIGS)

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libvplbm.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} is not built; run __graft_entry__.build() or "
                              "python -m paper_1905_05110_gb300.build")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise VplbmError(status, load_library().vplbm_last_error().decode())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


# ---- descriptors from problem dicts -------------------------------------------

def lattice_desc(problem: dict, precision: str = "f64", keep: list | None = None) -> LatticeDesc:
    """C lattice descriptor from a problem dict; ``keep`` receives array refs."""
    keep = keep if keep is not None else []
    d = LatticeDesc()
    d.nx, d.ny = int(problem["nx"]), int(problem["ny"])
    for k in range(9):
        d.s[k] = float(problem["s"][k])
    d.eta = float(problem.get("eta", 1e-3))
    d.rho0 = float(problem.get("rho0", 1.0))
    g = problem.get("g_fluid", (0.0, 0.0))
    d.gx, d.gy = float(g[0]), float(g[1])
    for k, side in enumerate(SIDES):
        bc = problem["bc"][side]
        d.bc[k].kind = BC_KINDS[bc["kind"]]
        u = bc.get("u", (0.0, 0.0))
        d.bc[k].ux, d.bc[k].uy = float(u[0]), float(u[1])
        for key, field in (("ux_profile", "ux_profile"), ("uy_profile", "uy_profile")):
            prof = bc.get(key)
            if prof is None:
                setattr(d.bc[k], field, None)
            else:
                arr = _f64(prof)
                keep.append(arr)
                setattr(d.bc[k], field, _dptr(arr))
    d.precision = PRECISIONS[precision]
    d.collision = COLLISIONS[problem.get("collision", "mrt")]
    return d


def body_desc(body: dict | None) -> BodyDesc | None:
    if not body:
        return None
    b = BodyDesc()
    b.radius = float(body["radius"])
    b.x, b.y = float(body["x"]), float(body["y"])
    b.theta = float(body.get("theta", 0.0))
    b.vx, b.vy = float(body.get("vx", 0.0)), float(body.get("vy", 0.0))
    b.omega = float(body.get("omega", 0.0))
    b.motion = MOTIONS[body.get("motion", "fixed")]
    b.axis = int(body.get("axis", 1))
    b.amp, b.freq = float(body.get("amp", 0.0)), float(body.get("freq", 0.0))
    b.phase = float(body.get("phase", 0.0))
    b.mass, b.inertia = float(body.get("mass", 1.0)), float(body.get("inertia", 1.0))
    for key in ("damp", "stiff", "q0", "f_ext"):
        vals = body.get(key, (0.0, 0.0, 0.0))
        arr = getattr(b, key)
        for k in range(3):
            arr[k] = float(vals[k])
    b.dof_mask = int(body.get("dof_mask", 0))
    b.u_ref, b.d_ref = float(body.get("u_ref", 0.0)), float(body.get("d_ref", 0.0))
    b.shape = SHAPES[body.get("shape", "disk")]
    b.radius_b = float(body.get("radius_b", body["radius"]))
    return b


def _byref(x):
    return None if x is None else C.byref(x)


# ---- same-name wrappers of the C entry points -----------------------------------

def vplbm_version() -> str:
    return load_library().vplbm_version().decode()


def vplbm_last_error() -> str:
    return load_library().vplbm_last_error().decode()


def vplbm_buffer_sizes_for(lat: LatticeDesc, body: BodyDesc | None, history_capacity: int) -> BufferSizes:
    out = BufferSizes()
    _check(load_library().vplbm_buffer_sizes_for(C.byref(lat), _byref(body), int(history_capacity),
                                                 C.byref(out)))
    return out


def vplbm_create(lat: LatticeDesc, body: BodyDesc | None, history_capacity: int, stream: int = 0):
    ctx = _CTX()
    _check(load_library().vplbm_create(C.byref(lat), _byref(body), int(history_capacity),
                                       C.c_void_p(stream), C.byref(ctx)))
    return ctx


def vplbm_create_with_buffers(lat: LatticeDesc, body: BodyDesc | None, history_capacity: int,
                              stream: int, buffers: Buffers):
    ctx = _CTX()
    _check(load_library().vplbm_create_with_buffers(C.byref(lat), _byref(body), int(history_capacity),
                                                    C.c_void_p(stream), C.byref(buffers), C.byref(ctx)))
    return ctx


def vplbm_create_bodies(lat: LatticeDesc, bodies: list, history_capacity: int, stream: int = 0):
    """Context with several bodies (a list of BodyDesc, 1 .. MAX_BODIES)."""
    arr = (BodyDesc * max(len(bodies), 1))(*bodies)
    ctx = _CTX()
    _check(load_library().vplbm_create_bodies(C.byref(lat), arr, len(bodies), int(history_capacity),
                                              C.c_void_p(stream), C.byref(ctx)))
    return ctx


def vplbm_destroy(ctx):
    load_library().vplbm_destroy(ctx)


def vplbm_init_equilibrium(ctx, rho=None, ux=None, uy=None):
    _check(load_library().vplbm_init_equilibrium(ctx, _dptr(rho), _dptr(ux), _dptr(uy)))


def vplbm_set_populations(ctx, f: np.ndarray):
    _check(load_library().vplbm_set_populations(ctx, _dptr(f)))


def vplbm_step(ctx, nsteps: int):
    _check(load_library().vplbm_step(ctx, int(nsteps)))


def vplbm_sync(ctx):
    _check(load_library().vplbm_sync(ctx))


def vplbm_get_populations(ctx, out: np.ndarray):
    _check(load_library().vplbm_get_populations(ctx, _dptr(out)))


def vplbm_get_fields(ctx, rho, ux, uy):
    _check(load_library().vplbm_get_fields(ctx, _dptr(rho), _dptr(ux), _dptr(uy)))


def vplbm_get_fields_dev(ctx, rho_ptr: int, ux_ptr: int, uy_ptr: int):
    _check(load_library().vplbm_get_fields_dev(ctx, C.c_void_p(rho_ptr), C.c_void_p(ux_ptr),
                                               C.c_void_p(uy_ptr)))


def vplbm_get_history(ctx, first: int, count: int):
    buf = (Record * max(int(count), 1))()
    _check(load_library().vplbm_get_history(ctx, int(first), int(count), buf))
    return buf


def vplbm_get_body(ctx):
    q = np.zeros(3)
    v = np.zeros(3)
    step = C.c_longlong()
    _check(load_library().vplbm_get_body(ctx, _dptr(q), _dptr(v), C.byref(step)))
    return q, v, int(step.value)


def vplbm_get_num_bodies(ctx) -> int:
    n = C.c_int()
    _check(load_library().vplbm_get_num_bodies(ctx, C.byref(n)))
    return int(n.value)


def vplbm_get_history_body(ctx, k: int, first: int, count: int):
    buf = (Record * max(int(count), 1))()
    _check(load_library().vplbm_get_history_body(ctx, int(k), int(first), int(count), buf))
    return buf


def vplbm_get_body_k(ctx, k: int):
    q = np.zeros(3)
    v = np.zeros(3)
    step = C.c_longlong()
    _check(load_library().vplbm_get_body_k(ctx, int(k), _dptr(q), _dptr(v), C.byref(step)))
    return q, v, int(step.value)


MAX_BODIES = 4   # VPLBM_MAX_BODIES


COLLISIONS = {"mrt": 0, "bgk": 1}
SHAPES = {"disk": 0, "ellipse": 1, "rectangle": 2}
BATCH_MODES = {"branches": 0, "tiles": 1, "persistent": 2}
BATCH_MODE_NAMES = {v: k for k, v in BATCH_MODES.items()}
KERNELS = {"scalar": 0, "scalar48": 1, "scalar40": 2, "tma": 3, "fused2": 4, "pair": 5}
KERNEL_NAMES = {v: k for k, v in KERNELS.items()}


def vplbm_set_launch(ctx, kernel: int, bx: int, by: int):
    _check(load_library().vplbm_set_launch(ctx, int(kernel), int(bx), int(by)))


def vplbm_get_launch(ctx):
    k, bx, by = C.c_int(), C.c_int(), C.c_int()
    _check(load_library().vplbm_get_launch(ctx, C.byref(k), C.byref(bx), C.byref(by)))
    return k.value, bx.value, by.value


def vplbm_autotune(ctx, steps_per_trial: int = 20):
    _check(load_library().vplbm_autotune(ctx, int(steps_per_trial)))


def vplbm_inject_wait_timeout(ctx, enable: bool):
    _check(load_library().vplbm_inject_wait_timeout(ctx, int(bool(enable))))


def vplbm_get_launch_count(ctx) -> int:
    n = C.c_longlong()
    _check(load_library().vplbm_get_launch_count(ctx, C.byref(n)))
    return int(n.value)


# Kinds of step-kernel launches (vplbm_launch_kind), in the order of the
# counts of vplbm_get_kernel_launches.
LAUNCH_KINDS = ("one_step", "two_step", "lookahead", "tma")


def vplbm_get_kernel_launches(ctx) -> dict:
    counts = (C.c_longlong * len(LAUNCH_KINDS))()
    _check(load_library().vplbm_get_kernel_launches(ctx, counts))
    return {k: int(counts[n]) for n, k in enumerate(LAUNCH_KINDS)}


def vplbm_eval_recip_f32(x_ptr: int, y_ptr: int, n: int, stream: int = 0):
    """y[k] := the step kernels' FP32 reciprocal of x[k] (device arrays)."""
    _check(load_library().vplbm_eval_recip_f32(C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(n), C.c_void_p(stream)))


def vplbm_step_noalloc(lat: LatticeDesc, body: BodyDesc | None, populations_ptrs, state_ptr: int,
                       history_ptr: int | None, history_capacity: int, nsteps: int, stream: int = 0):
    """Allocation-free steps on caller-owned device buffers (see include/vplbm.h)."""
    pops = (C.c_void_p * 2)(int(populations_ptrs[0]), int(populations_ptrs[1]))
    _check(load_library().vplbm_step_noalloc(C.byref(lat), _byref(body), pops, C.c_void_p(state_ptr),
                                             C.c_void_p(history_ptr or 0), int(history_capacity),
                                             int(nsteps), C.c_void_p(stream)))


def vplbm_batch_create(lats, bodies, history_capacity: int, stream: int = 0):
    """lats: list of LatticeDesc; bodies: list of BodyDesc or None per member."""
    n = len(lats)
    lat_arr = (LatticeDesc * n)(*lats)
    body_ptrs = (C.POINTER(BodyDesc) * n)(*[C.pointer(b) if b is not None else C.POINTER(BodyDesc)()
                                            for b in bodies])
    out = C.c_void_p()
    _check(load_library().vplbm_batch_create(lat_arr, C.cast(body_ptrs, C.c_void_p), n, int(history_capacity),
                                             C.c_void_p(stream), C.byref(out)))
    return out


def vplbm_batch_destroy(batch):
    load_library().vplbm_batch_destroy(batch)


def vplbm_batch_member(batch, k: int):
    ctx = _CTX()
    _check(load_library().vplbm_batch_member(batch, int(k), C.byref(ctx)))
    return ctx


def vplbm_batch_step(batch, nsteps: int):
    _check(load_library().vplbm_batch_step(batch, int(nsteps)))


def vplbm_batch_sync(batch):
    _check(load_library().vplbm_batch_sync(batch))


def vplbm_batch_set_launch(batch, block_x: int, block_y: int = 1, tiles_per_block: int = 1):
    _check(load_library().vplbm_batch_set_launch(batch, int(block_x), int(block_y), int(tiles_per_block)))


def vplbm_batch_get_launch(batch):
    bx, by, rows, n = C.c_int(), C.c_int(), C.c_int(), C.c_longlong()
    _check(load_library().vplbm_batch_get_launch(batch, C.byref(bx), C.byref(by), C.byref(rows), C.byref(n)))
    return bx.value, by.value, rows.value, int(n.value)


def vplbm_batch_set_mode(batch, mode: int):
    _check(load_library().vplbm_batch_set_mode(batch, int(mode)))


def vplbm_batch_get_mode(batch) -> int:
    m = C.c_int()
    _check(load_library().vplbm_batch_get_mode(batch, C.byref(m)))
    return m.value


def vplbm_batch_autotune(batch, steps_per_trial: int = 8):
    _check(load_library().vplbm_batch_autotune(batch, int(steps_per_trial)))


def vplbm_batch_set_persistent(batch, block_x: int = 64, block_y: int = 4, chunk: int = 2,
                               params_in_shared: bool = False):
    _check(load_library().vplbm_batch_set_persistent(batch, int(block_x), int(block_y), int(chunk),
                                                     int(bool(params_in_shared))))


def vplbm_batch_get_persistent(batch):
    """(block_x, block_y, chunk, params_in_shared, grid, persistent launches so far)."""
    v = [C.c_int() for _ in range(5)]
    n = C.c_longlong()
    _check(load_library().vplbm_batch_get_persistent(batch, *[C.byref(x) for x in v], C.byref(n)))
    return tuple(x.value for x in v) + (int(n.value),)


def vplbm_batch_inject_barrier_timeout(batch, enable: bool):
    _check(load_library().vplbm_batch_inject_barrier_timeout(batch, int(bool(enable))))


def vplbm_adjoint(ctx, ny: int, nsteps: int, window_start: int, w_cd: float = 1.0, w_cl: float = 0.0,
                  checkpoint_interval: int = 0):
    """Discrete-adjoint gradient; returns (grad[ny + 3], (J1, J2))."""
    d = AdjointDesc(int(nsteps), int(window_start), float(w_cd), float(w_cl), int(checkpoint_interval))
    grad = np.zeros(int(ny) + 3)
    js = np.zeros(2)
    _check(load_library().vplbm_adjoint(ctx, C.cast(C.pointer(d), C.c_void_p), _dptr(grad), _dptr(js)))
    return grad, (float(js[0]), float(js[1]))


def vplbm_save(ctx, path: str):
    _check(load_library().vplbm_save(ctx, os.fsencode(path)))


def vplbm_load(ctx, path: str):
    _check(load_library().vplbm_load(ctx, os.fsencode(path)))


# ---- convenience object ------------------------------------------------------------

class Simulation:
    """One VP-LBM simulation on the current CUDA device.

    Device buffers are torch tensors handed to ``vplbm_create_with_buffers``;
    work runs on ``stream`` (default: torch's current stream).  A problem
    with a "bodies" list of two or more bodies is created with
    ``vplbm_create_bodies`` (the library allocates its memory).
    """

    def __init__(self, problem: dict, precision: str = "f32", history_capacity: int = 1 << 16,
                 stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Simulation needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.problem = problem
        self.precision = precision
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])
        self._keep: list = []
        self._lat = lattice_desc(problem, precision, self._keep)
        bodies = list(problem["bodies"]) if problem.get("bodies") else (
            [problem["body"]] if problem.get("body") else [])
        self.nbodies = len(bodies)
        self.history_capacity = int(history_capacity)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        if len(bodies) > 1:
            self._bodies = [body_desc(b) for b in bodies]
            self.ctx = vplbm_create_bodies(self._lat, self._bodies, self.history_capacity,
                                           self.stream.cuda_stream)
            return
        self._body = body_desc(bodies[0] if bodies else None)
        sizes = vplbm_buffer_sizes_for(self._lat, self._body, self.history_capacity)
        self._tensors = {}

        def alloc(name, nbytes):
            # one extra 256-byte slot so the data pointer can be aligned
            t = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
            self._tensors[name] = t
            ptr = t.data_ptr()
            return ptr + (-ptr) % 256

        bufs = Buffers()
        bufs.populations_dev[0] = alloc("f0", sizes.populations)
        bufs.populations_dev[1] = alloc("f1", sizes.populations)
        bufs.body_state_dev = alloc("bs", sizes.body_state)
        bufs.partials_dev = alloc("partials", sizes.partials)
        bufs.history_dev = alloc("hist", sizes.history)
        bufs.profiles_dev = alloc("prof", sizes.profiles)
        bufs.control_dev = alloc("ctrl", sizes.control)
        self.ctx = vplbm_create_with_buffers(self._lat, self._body, self.history_capacity,
                                             self.stream.cuda_stream, bufs)

    def close(self):
        """Destroy the context (device memory it owns, graphs, the adjoint workspace)."""
        if getattr(self, "ctx", None):
            vplbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state -------------------------------------------------------------------------
    def init_equilibrium(self, rho=None, ux=None, uy=None):
        """Equilibrium populations (Eq. 11) of host fields rho, ux, uy ([ny, nx],
        FP64; None: rho0 and 0); resets the step counter and the body."""
        shape = (self.ny, self.nx)
        arrs = [None if a is None else _f64(np.broadcast_to(a, shape)) for a in (rho, ux, uy)]
        vplbm_init_equilibrium(self.ctx, *arrs)

    def init_from_problem(self):
        """Equilibrium of the problem's uniform initial state."""
        init = self.problem.get("init", {})
        u = init.get("u", (0.0, 0.0))
        self.init_equilibrium(init.get("rho", None), u[0], u[1])

    def set_populations(self, f):
        """Set the full populations f[9, ny, nx] (FP64, host); stored in the context's precision."""
        vplbm_set_populations(self.ctx, _f64(f, (Q, self.ny, self.nx)))

    def step(self, n: int = 1):
        """Advance n time steps (asynchronous on the simulation's stream)."""
        vplbm_step(self.ctx, n)

    def sync(self):
        """Wait for the stream; raises VplbmError on a latched device error (non-finite density, a timed-out wait)."""
        vplbm_sync(self.ctx)

    def populations(self) -> np.ndarray:
        """The full populations f[9, ny, nx] in FP64 (deviation storage has w rho0 added back)."""
        out = np.empty((Q, self.ny, self.nx))
        vplbm_get_populations(self.ctx, out)
        return out

    def fields(self):
        """rho, ux, uy [ny, nx] in FP64 at the current step."""
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        vplbm_get_fields(self.ctx, rho, ux, uy)
        return rho, ux, uy

    def history(self, first: int = 0, count: int | None = None, body: int = 0) -> np.ndarray:
        """Records [first, first + count) of body `body`, one row per step."""
        if count is None:
            count = self.nstep - first
        buf = vplbm_get_history_body(self.ctx, body, first, count)
        arr = np.frombuffer(buf, dtype=np.float64, count=count * len(RECORD_FIELDS))
        return arr.reshape(count, len(RECORD_FIELDS)).copy()

    def body_state(self, body: int = 0):
        """Pose (x_G, y_G, theta) and velocity (vx, vy, omega) of body `body` at the current step."""
        q, v, _ = vplbm_get_body_k(self.ctx, body)
        return q, v

    @property
    def nstep(self) -> int:
        """Time steps taken since the last initialisation."""
        return vplbm_get_body(self.ctx)[2]

    def set_launch(self, kernel, bx=0, by=0):
        """kernel: "scalar" (64-register budget), "scalar48", "scalar40", "tma", "fused2"
        (two steps per launch; bx, by: the blocks of its single steps) or "pair" (two
        nodes per thread, FP16 storage) (or its number)."""
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        vplbm_set_launch(self.ctx, k, bx, by)

    def launch(self):
        """(kernel name, block_x, block_y) of the step kernel."""
        k, bx, by = vplbm_get_launch(self.ctx)
        return KERNEL_NAMES[k], bx, by

    def autotune(self, steps_per_trial: int = 20):
        """Time the step kernels and launch shapes over short trials, keep the fastest; returns it as launch()."""
        vplbm_autotune(self.ctx, steps_per_trial)
        return self.launch()

    @property
    def launches(self) -> int:
        """Kernel launches made by step() since creation."""
        return vplbm_get_launch_count(self.ctx)

    def kernel_launches(self) -> dict:
        """Launches made so far by kind: one_step, two_step, lookahead, tma."""
        return vplbm_get_kernel_launches(self.ctx)

    def adjoint(self, nsteps: int, window_start: int, w_cd: float = 1.0, w_cl: float = 0.0,
                checkpoint_interval: int = 0):
        """Gradient of w_cd mean C_D + w_cl RMS C_L over [window_start, nsteps)
        of a run of nsteps steps from the current state, with respect to the
        west inlet profile (ny values), eta, s_nu and s_e; returns (grad, (J1, J2)).
        The context ends at the state after the forward run, and keeps the
        adjoint's device workspace for later calls until close()."""
        return vplbm_adjoint(self.ctx, self.ny, nsteps, window_start, w_cd, w_cl, checkpoint_interval)

    def save(self, path):
        """Write a checkpoint (populations, body state, step counter, history ring) to path."""
        vplbm_save(self.ctx, path)

    def load(self, path):
        """Read a checkpoint written by save() on a context of the same size, precision and history capacity."""
        vplbm_load(self.ctx, path)


class _Member:
    """A batch member: the per-simulation calls on a context the batch owns."""

    def __init__(self, ctx, problem):
        self.ctx = ctx
        self.problem = problem
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])

    init_equilibrium = Simulation.init_equilibrium
    init_from_problem = Simulation.init_from_problem
    set_populations = Simulation.set_populations
    populations = Simulation.populations
    fields = Simulation.fields
    history = Simulation.history
    body_state = Simulation.body_state
    nstep = Simulation.nstep
    launch = Simulation.launch


class Batch:
    """Many simulations of uneven sizes stepped together: concurrent graph
    branches (one per member), one launch per step over all members' tiles,
    or one persistent launch for many steps (set_mode, autotune)."""

    def __init__(self, problems, precision: str = "f32", history_capacity: int = 1 << 12, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device; there is no CPU fallback")
        self.problems = list(problems)
        self._keep: list = []
        lats = [lattice_desc(p, precision, self._keep) for p in self.problems]
        bodies = [body_desc(p.get("body")) for p in self.problems]
        self._bodies = bodies
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = vplbm_batch_create(lats, bodies, history_capacity, self.stream.cuda_stream)
        self.members = [_Member(vplbm_batch_member(self.handle, k), p) for k, p in enumerate(self.problems)]

    def close(self):
        """Destroy the batch and every member's context."""
        if getattr(self, "handle", None):
            vplbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_from_problems(self):
        """Every member at the equilibrium of its problem's uniform initial state."""
        for m in self.members:
            m.init_from_problem()

    def step(self, n: int = 1):
        """Advance every member n time steps (asynchronous on the batch's stream)."""
        vplbm_batch_step(self.handle, n)

    def sync(self):
        """Wait for the stream; raises VplbmError on a latched device error of any member
        (a persistent launch's timed-out grid barrier included)."""
        vplbm_batch_sync(self.handle)

    def set_launch(self, block_x: int, block_y: int = 1, tiles_per_block: int = 1):
        """Block shape and tiles per block of the one-launch-per-step (tile) mode."""
        vplbm_batch_set_launch(self.handle, block_x, block_y, tiles_per_block)

    def launch(self):
        """(block_x, block_y, tiles_per_block, batched launches so far)."""
        return vplbm_batch_get_launch(self.handle)

    def set_mode(self, mode):
        """"branches" (each member's own kernel, concurrent graph branches), "tiles" (one
        launch per step) or "persistent" (one launch for many steps)."""
        vplbm_batch_set_mode(self.handle, BATCH_MODES[mode] if isinstance(mode, str) else int(mode))

    @property
    def mode(self) -> str:
        """The current mode: "branches", "tiles" or "persistent"."""
        return BATCH_MODE_NAMES[vplbm_batch_get_mode(self.handle)]

    def set_persistent(self, block_x: int = 64, block_y: int = 4, chunk: int = 2, params_in_shared: bool = False):
        """Block shape, work items per queue draw and parameter staging of the persistent mode."""
        vplbm_batch_set_persistent(self.handle, block_x, block_y, chunk, params_in_shared)

    def persistent(self):
        """(block_x, block_y, chunk, params_in_shared, grid, persistent launches so far)."""
        return vplbm_batch_get_persistent(self.handle)

    def inject_barrier_timeout(self, enable: bool = True):
        """Test hook: the persistent launch's grid barriers wait for one arrival more than
        the grid makes, so they give up after a short bounded wait (ETIMEOUT at sync)."""
        vplbm_batch_inject_barrier_timeout(self.handle, enable)

    def autotune(self, steps_per_trial: int = 8):
        """Fastest of the branch mode, the tile-mode shapes and the persistent variants:
        (mode, block_x, block_y, tiles_per_block) or, persistent,
        (mode, block_x, block_y, chunk, params_in_shared)."""
        vplbm_batch_autotune(self.handle, steps_per_trial)
        if self.mode == "persistent":
            return (self.mode,) + tuple(self.persistent()[:4])
        return (self.mode,) + tuple(self.launch()[:3])
