"""Plain FP64 CPU oracle of the VP-LBM step (test infrastructure only).

Only the test-suite, the package smoke check and the CPU-baseline leg of the
benchmark may import this module.  It wraps ``vplbm_oracle.c`` (compiled with
gcc, ``-ffp-contract=off``) through ctypes and shares nothing with the CUDA
implementation: its own descriptors, its own constants, its own build.

Problem descriptions are plain dicts (see ``workloads.py`` at the repository
root for the keys); this module turns them into the oracle's own C structs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vplbm_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
# VPLBM_ORACLE_PLANT=k (k > 0) loads the oracle built with planted mistake k
# into a library of its own (the test of the pins); unset or 0: the oracle.
PLANT = int(os.environ.get("VPLBM_ORACLE_PLANT", "0") or 0)
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so" if PLANT == 0 else f"liboracle_plant{PLANT}.so")

Q = 9
BC_KINDS = {"periodic": 0, "noslip": 1, "velocity": 2, "zerograd": 3, "symmetry": 4, "convective": 5}
MOTIONS = {"fixed": 0, "imposed": 1, "free": 2}
SIDES = ("west", "east", "south", "north")
RECORD_FIELDS = ("t", "fx", "fy", "torque", "cd", "cl", "x", "y", "theta",
                 "vx", "vy", "omega", "fpen_x", "fpen_y", "tpen", "n_solid")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, plain C99)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"] + ([f"-DORACLE_PLANT={PLANT}"] if PLANT else [])
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("s", C.c_double * Q), ("eta", C.c_double), ("rho0", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double),
                ("bc_kind", C.c_int * 4), ("bc_u", (C.c_double * 2) * 4),
                ("bc_ux", C.POINTER(C.c_double) * 4), ("bc_uy", C.POINTER(C.c_double) * 4),
                ("collision", C.c_int)]


COLLISIONS = {"mrt": 0, "bgk": 1}


class Body(C.Structure):
    _fields_ = [("present", C.c_int), ("radius", C.c_double),
                ("x", C.c_double), ("y", C.c_double), ("theta", C.c_double),
                ("vx", C.c_double), ("vy", C.c_double), ("omega", C.c_double),
                ("motion", C.c_int), ("axis", C.c_int),
                ("amp", C.c_double), ("freq", C.c_double), ("phase", C.c_double),
                ("mass", C.c_double), ("inertia", C.c_double),
                ("damp", C.c_double * 3), ("stiff", C.c_double * 3),
                ("q0", C.c_double * 3), ("f_ext", C.c_double * 3),
                ("dof_mask", C.c_uint), ("u_ref", C.c_double), ("d_ref", C.c_double),
                ("shape", C.c_int), ("radius_b", C.c_double)]


SHAPES = {"disk": 0, "ellipse": 1, "rectangle": 2}


class Record(C.Structure):
    _fields_ = [(n, C.c_double) for n in RECORD_FIELDS]


class AdjointDesc(C.Structure):
    _fields_ = [("nsteps", C.c_longlong), ("w0", C.c_longlong), ("w_cd", C.c_double), ("w_cl", C.c_double)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(Lattice), C.POINTER(Body), C.c_longlong]
            L.orc_create_bodies.restype = C.c_void_p
            L.orc_create_bodies.argtypes = [C.POINTER(Lattice), C.POINTER(Body), C.c_int, C.c_longlong]
            L.orc_get_history_body.restype = C.c_int
            L.orc_get_history_body.argtypes = [C.c_void_p, C.c_int, C.c_longlong, C.c_longlong, C.POINTER(Record)]
            L.orc_get_body_k.argtypes = [C.c_void_p, C.c_int, _D, _D]
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_init_equilibrium.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_set_populations.argtypes = [C.c_void_p, _D]
            L.orc_get_populations.argtypes = [C.c_void_p, _D]
            L.orc_get_fields.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_step.argtypes = [C.c_void_p, C.c_longlong]
            L.orc_get_step.restype = C.c_longlong
            L.orc_get_step.argtypes = [C.c_void_p]
            L.orc_get_history.restype = C.c_int
            L.orc_get_history.argtypes = [C.c_void_p, C.c_longlong, C.c_longlong, C.POINTER(Record)]
            L.orc_get_body.argtypes = [C.c_void_p, _D, _D]
            L.orc_constants.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, _D]
            L.orc_moment_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, _D]
            L.orc_guo_forcing.argtypes = [C.c_double] * 4 + [_D]
            L.orc_collide.argtypes = [_D, _D] + [C.c_double] * 5 + [_D]
            L.orc_collide_bgk.argtypes = [_D] + [C.c_double] * 6 + [_D]
            L.orc_penalized_velocity.argtypes = ([C.c_double] * 3 + [C.c_int]
                                                 + [C.c_double] * 5 + [_D])
            L.orc_body_advance.argtypes = [C.POINTER(Body), C.c_longlong, C.c_double,
                                           _D, _D, _D]
            L.orc_chi.restype = C.c_int
            L.orc_chi.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_adjoint.restype = C.c_int
            L.orc_adjoint.argtypes = [C.c_void_p, C.POINTER(AdjointDesc), _D, _D]
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_lattice(p: dict, keep: list) -> Lattice:
    """Oracle lattice struct from a problem dict; ``keep`` holds array refs."""
    lat = Lattice()
    lat.nx, lat.ny = int(p["nx"]), int(p["ny"])
    for k in range(Q):
        lat.s[k] = float(p["s"][k])
    lat.eta = float(p.get("eta", 1e-3))
    lat.rho0 = float(p.get("rho0", 1.0))
    lat.collision = COLLISIONS[p.get("collision", "mrt")]
    g = p.get("g_fluid", (0.0, 0.0))
    lat.gx, lat.gy = float(g[0]), float(g[1])
    bcs = p["bc"]
    for side_i, side in enumerate(SIDES):
        bc = bcs[side]
        lat.bc_kind[side_i] = BC_KINDS[bc["kind"]]
        u = bc.get("u", (0.0, 0.0))
        lat.bc_u[side_i][0], lat.bc_u[side_i][1] = float(u[0]), float(u[1])
        for comp, key in ((0, "ux_profile"), (1, "uy_profile")):
            prof = bc.get(key)
            ptr = None
            if prof is not None:
                arr = _f64(prof)
                n_edge = lat.ny if side_i < 2 else lat.nx
                if arr.shape != (n_edge,):
                    raise ValueError(f"{side}.{key}: expected {n_edge} values")
                keep.append(arr)
                ptr = _dptr(arr)
            if comp == 0:
                lat.bc_ux[side_i] = ptr
            else:
                lat.bc_uy[side_i] = ptr
    return lat


def make_body(b: dict | None) -> Body:
    body = Body()
    if not b:
        body.present = 0
        return body
    body.present = 1
    body.radius = float(b["radius"])
    body.x, body.y = float(b["x"]), float(b["y"])
    body.theta = float(b.get("theta", 0.0))
    body.vx, body.vy = float(b.get("vx", 0.0)), float(b.get("vy", 0.0))
    body.omega = float(b.get("omega", 0.0))
    body.motion = MOTIONS[b.get("motion", "fixed")]
    body.axis = int(b.get("axis", 1))
    body.amp = float(b.get("amp", 0.0))
    body.freq = float(b.get("freq", 0.0))
    body.phase = float(b.get("phase", 0.0))
    body.mass = float(b.get("mass", 1.0))
    body.inertia = float(b.get("inertia", 1.0))
    for key in ("damp", "stiff", "q0", "f_ext"):
        vals = b.get(key, (0.0, 0.0, 0.0))
        arr = getattr(body, key)
        for d in range(3):
            arr[d] = float(vals[d])
    body.dof_mask = int(b.get("dof_mask", 0))
    body.u_ref = float(b.get("u_ref", 0.0))
    body.d_ref = float(b.get("d_ref", 0.0))
    body.shape = SHAPES[b.get("shape", "disk")]
    body.radius_b = float(b.get("radius_b", b["radius"]))
    return body


def problem_bodies(problem: dict) -> list:
    """The bodies of a problem: its "bodies" list, or its single "body"."""
    if problem.get("bodies"):
        return list(problem["bodies"])
    return [problem["body"]] if problem.get("body") else []


class OracleSim:
    """One FP64 VP-LBM simulation on the CPU (plain loops, Algorithm 1)."""

    def __init__(self, problem: dict, hist_cap: int = 1 << 16):
        L = lib()
        self.p = problem
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])
        self._keep: list = []
        self._lat = make_lattice(problem, self._keep)
        bodies = problem_bodies(problem)
        self.nbodies = len(bodies)
        self._bodies = (Body * max(1, len(bodies)))(*[make_body(b) for b in bodies])
        self._h = L.orc_create_bodies(C.byref(self._lat), self._bodies, len(bodies), int(hist_cap))
        if not self._h:
            raise ValueError("oracle: invalid lattice")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def init_equilibrium(self, rho=None, ux=None, uy=None):
        shape = (self.ny, self.nx)
        args = []
        for a in (rho, ux, uy):
            if a is None:
                args.append(None)
            else:
                arr = _f64(a).reshape(shape)
                self._keep.append(arr)
                args.append(_dptr(arr))
        lib().orc_init_equilibrium(self._h, *args)

    def set_populations(self, f):
        arr = _f64(f).reshape(Q, self.ny, self.nx)
        lib().orc_set_populations(self._h, _dptr(arr))

    def populations(self) -> np.ndarray:
        out = np.empty((Q, self.ny, self.nx))
        lib().orc_get_populations(self._h, _dptr(out))
        return out

    def fields(self):
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        lib().orc_get_fields(self._h, _dptr(rho), _dptr(ux), _dptr(uy))
        return rho, ux, uy

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def nstep(self) -> int:
        return int(lib().orc_get_step(self._h))

    def history(self, first: int = 0, count: int | None = None, body: int = 0) -> np.ndarray:
        if count is None:
            count = self.nstep - first
        buf = (Record * max(count, 1))()
        if lib().orc_get_history_body(self._h, int(body), first, count, buf) != 0:
            raise IndexError("oracle history range not available")
        out = np.zeros((count, len(RECORD_FIELDS)))
        for k in range(count):
            out[k] = [getattr(buf[k], n) for n in RECORD_FIELDS]
        return out

    def adjoint(self, nsteps: int, w0: int, w_cd: float = 1.0, w_cl: float = 0.0):
        """Forward nsteps from the current state, then the discrete adjoint.

        Returns (grad, (J1, J2)); grad = [dJ/du_in(j) for the west wall's u_x
        profile (ny values)] + [dJ/deta, dJ/ds_nu, dJ/ds_e] for
        J = w_cd * mean C_D + w_cl * RMS C_L over steps [w0, nsteps).
        """
        d = AdjointDesc(int(nsteps), int(w0), float(w_cd), float(w_cl))
        grad = np.zeros(self.ny + 3)
        js = np.zeros(2)
        if lib().orc_adjoint(self._h, C.byref(d), _dptr(grad), _dptr(js)) != 0:
            raise ValueError("oracle adjoint: free body or history ring too short")
        return grad, (float(js[0]), float(js[1]))

    def body_state(self, body: int = 0):
        q = np.zeros(3)
        v = np.zeros(3)
        lib().orc_get_body_k(self._h, int(body), _dptr(q), _dptr(v))
        return q, v

    def chi(self) -> np.ndarray:
        """chi of every node at the current pose, [ny, nx] (0 / 1)."""
        out = np.zeros((self.ny, self.nx), dtype=np.int8)
        L = lib()
        for j in range(self.ny):
            for i in range(self.nx):
                out[j, i] = L.orc_chi(self._h, i, j)
        return out


# ---- single-node functions (for pinning the oracle) -------------------------

def constants():
    c = np.zeros((Q, 2), dtype=np.int32)
    w = np.zeros(Q)
    m = np.zeros((Q, Q))
    minv = np.zeros((Q, Q))
    lib().orc_constants(c.ctypes.data_as(C.c_void_p), _dptr(w), _dptr(m), _dptr(minv))
    return c, w, m, minv


def equilibrium(rho, ux, uy) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_equilibrium(rho, ux, uy, _dptr(out))
    return out


def moment_equilibrium(rho, ux, uy) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_moment_equilibrium(rho, ux, uy, _dptr(out))
    return out


def guo_forcing(ux, uy, gx, gy) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_guo_forcing(ux, uy, gx, gy, _dptr(out))
    return out


def collide(f, s, rho, ux, uy, gx, gy) -> np.ndarray:
    f = _f64(f)
    s = _f64(s)
    out = np.zeros(Q)
    lib().orc_collide(_dptr(f), _dptr(s), rho, ux, uy, gx, gy, _dptr(out))
    return out


def collide_bgk(f, omega, rho, ux, uy, gx, gy) -> np.ndarray:
    """BGK collision of Sec. 2.1 with the Eq. (12) forcing (rate omega = 1/tau)."""
    f = _f64(f)
    out = np.zeros(Q)
    lib().orc_collide_bgk(_dptr(f), omega, rho, ux, uy, gx, gy, _dptr(out))
    return out


def penalized_velocity(rho, jx, jy, chi, usx, usy, eta, gx=0.0, gy=0.0):
    out = np.zeros(4)
    lib().orc_penalized_velocity(rho, jx, jy, int(chi), usx, usy, eta, gx, gy, _dptr(out))
    return out  # ux, uy, ax, ay


def body_advance(body: dict, step: int, q_center: float, F, q, v):
    b = make_body(body)
    F = _f64(F).copy()
    q = _f64(q).copy()
    v = _f64(v).copy()
    lib().orc_body_advance(C.byref(b), int(step), float(q_center), _dptr(F), _dptr(q), _dptr(v))
    return q, v
