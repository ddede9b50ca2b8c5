"""Python binding of the C ABI in include/sph.h (argument marshalling only).

Every step of the method runs in the CUDA library ``libsph_gb300.so``; this
module converts numpy arrays to pointers, calls the C functions by the same
names, and turns status codes into exceptions.  There is no fallback: if
the library is missing or cannot load, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_ECAPACITY, SPH_ENONFINITE, \
    SPH_ETIMEOUT, SPH_ESTATE = range(8)
STATUS_NAMES = ["SPH_OK", "SPH_EINVAL", "SPH_ENOMEM", "SPH_ECUDA",
                "SPH_ECAPACITY", "SPH_ENONFINITE", "SPH_ETIMEOUT",
                "SPH_ESTATE"]
SPH_FLUID, SPH_WALL, SPH_BACKGROUND, SPH_REGION = 0, 1, 2, 3
SPH_FP64, SPH_MIXED = 0, 1
SPH_READ_BY_ID = 0x100

FIELDS = ["x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax", "id",
          "beta", "pavg", "drx", "dry", "dpdt", "dudt", "dvdt", "nnb",
          "cellkey", "neigh_off", "neigh_id", "omega",
          "bg_x", "bg_y", "bg_h", "bg_m", "bg_ds", "bg_id"]
FIELD = {k: i for i, k in enumerate(FIELDS)}
_FIELD_DTYPE = {"id": np.int64, "nnb": np.int32, "cellkey": np.uint64,
                "neigh_off": np.int64, "neigh_id": np.int64,
                "bg_id": np.int64}

TIMER_PASS_B, TIMER_PASS_A, TIMER_REBUILD, TIMER_PEC, TIMER_ADAPT, \
    TIMER_WALK, TIMER_SORT = range(7)


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8
                                     else status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
        ("periodic", ctypes.c_int * 2),
        ("rho0", ctypes.c_double), ("cs", ctypes.c_double),
        ("nu", ctypes.c_double), ("U_ref", ctypes.c_double),
        ("hdx", ctypes.c_double), ("alpha_e", ctypes.c_double),
        ("split_alpha", ctypes.c_double), ("split_eps", ctypes.c_double),
        ("Cr", ctypes.c_double), ("ds_min", ctypes.c_double),
        ("ds_max", ctypes.c_double),
        ("merge_iters", ctypes.c_int), ("shift_iters", ctypes.c_int),
        ("precision", ctypes.c_int), ("capacity", ctypes.c_longlong),
        ("pavg_mode", ctypes.c_int), ("edac_diff_denominator", ctypes.c_int),
        ("edac_rho_factor", ctypes.c_int), ("cell_c0", ctypes.c_double),
        ("bg_Nr", ctypes.c_double), ("bg_smooth_iters", ctypes.c_int),
        ("vort_k", ctypes.c_double), ("n_bg", ctypes.c_int),
        ("bg_capacity", ctypes.c_longlong),
        ("sponge_width", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)


class Tune(ctypes.Structure):
    """sph_tune: launch configuration of a context (sph.h)."""
    _fields_ = [("cell_scale", ctypes.c_double), ("walk", ctypes.c_int),
                ("team_a", ctypes.c_int), ("team_b", ctypes.c_int),
                ("walls", ctypes.c_int), ("no_graphs", ctypes.c_int),
                ("ms_cell", ctypes.c_double * 3),
                ("ms_walk", ctypes.c_double * 3),
                ("ms_team_a", ctypes.c_double * 4),
                ("ms_team_b", ctypes.c_double * 4),
                ("ms_walls", ctypes.c_double * 2)]


class Particles(ctypes.Structure):
    _fields_ = [(k, _D) for k in ("x", "y", "u", "v", "p", "rho", "m", "h",
                                  "mmin", "mmax", "ds")] + [
        ("id", ctypes.POINTER(ctypes.c_int64))]


class AdaptStats(ctypes.Structure):
    _fields_ = [("n_before", ctypes.c_longlong), ("n_split", ctypes.c_longlong),
                ("n_merged", ctypes.c_longlong), ("n_after", ctypes.c_longlong),
                ("mass_before", ctypes.c_double),
                ("mass_after", ctypes.c_double),
                ("n_bg_nearest", ctypes.c_longlong)]


class BgStats(ctypes.Structure):
    _fields_ = [("n_before", ctypes.c_longlong), ("n_marked", ctypes.c_longlong),
                ("n_vort", ctypes.c_longlong), ("n_split", ctypes.c_longlong),
                ("n_after", ctypes.c_longlong), ("iterations", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_longlong), ("n_wall", ctypes.c_longlong),
                ("n_bg", ctypes.c_longlong), ("t", ctypes.c_double),
                ("dt", ctypes.c_double), ("c0", ctypes.c_double),
                ("levels", ctypes.c_int), ("steps", ctypes.c_longlong),
                ("launches", ctypes.c_longlong),
                ("next_id", ctypes.c_longlong),
                ("n_region", ctypes.c_longlong),
                ("graph_steps", ctypes.c_longlong)]


_lib = None


def lib(build_if_missing: bool = True):
    """Load libsph_gb300.so (building it first if asked and needed); with
    SPH_GB300_DEBUG_LIB=1 in the environment, the debug build with device
    bounds checks (libsph_gb300_debug.so) instead."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("SPH_GB300_DEBUG_LIB") == "1"
    path = _build.LIB_DEBUG if debug else _build.LIB
    if build_if_missing:
        path = _build.build(debug=debug)
    if not os.path.exists(path):
        raise OSError("libsph_gb300.so not built: %s" % path)
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    ctx = ctypes.c_void_p
    L.sph_default_params.restype = None
    L.sph_default_params.argtypes = [P(Params)]
    L.sph_create.restype = ctypes.c_int
    L.sph_create.argtypes = [P(Params), ctypes.c_void_p, P(ctx)]
    L.sph_load_particles.restype = ctypes.c_int
    L.sph_load_particles.argtypes = [ctx, ctypes.c_int, ctypes.c_longlong,
                                     P(Particles)]
    L.sph_rhs.restype = ctypes.c_int
    L.sph_rhs.argtypes = [ctx]
    L.sph_step.restype = ctypes.c_int
    L.sph_step.argtypes = [ctx, ctypes.c_int, _D]
    L.sph_adapt.restype = ctypes.c_int
    L.sph_adapt.argtypes = [ctx, P(AdaptStats)]
    L.sph_background.restype = ctypes.c_int
    L.sph_background.argtypes = [ctx, ctypes.c_int, P(BgStats)]
    L.sph_autotune.restype = ctypes.c_int
    L.sph_autotune.argtypes = [ctx, P(Tune)]
    L.sph_set_tuning.restype = ctypes.c_int
    L.sph_set_tuning.argtypes = [ctx, P(Tune)]
    L.sph_forces.restype = ctypes.c_int
    L.sph_forces.argtypes = [ctx, ctypes.c_void_p, _D]
    L.sph_read.restype = ctypes.c_int
    L.sph_read.argtypes = [ctx, ctypes.c_int, ctypes.c_void_p,
                           ctypes.c_longlong, P(ctypes.c_longlong)]
    L.sph_get_info.restype = ctypes.c_int
    L.sph_get_info.argtypes = [ctx, P(Info)]
    L.sph_set_timing.restype = ctypes.c_int
    L.sph_set_timing.argtypes = [ctx, ctypes.c_int]
    L.sph_kernel_time.restype = ctypes.c_int
    L.sph_kernel_time.argtypes = [ctx, ctypes.c_int, _D,
                                  P(ctypes.c_longlong), ctypes.c_int]
    L.sph_destroy.restype = ctypes.c_int
    L.sph_destroy.argtypes = [ctx]
    L.sph_last_error.restype = ctypes.c_char_p
    L.sph_last_error.argtypes = [ctx]
    L.sph_cell_sort_noalloc.restype = ctypes.c_int
    L.sph_cell_sort_noalloc.argtypes = [P(Params), ctypes.c_longlong] + \
        [ctypes.c_void_p] * 6
    L.sph_batch_create.restype = ctypes.c_int
    L.sph_batch_create.argtypes = [ctypes.c_int, ctypes.c_void_p, P(ctypes.c_void_p)]
    L.sph_batch_destroy.restype = ctypes.c_int
    L.sph_batch_destroy.argtypes = [ctypes.c_void_p]
    L.sph_batch_step.restype = ctypes.c_int
    L.sph_batch_step.argtypes = [ctypes.c_void_p, P(ctypes.c_void_p), ctypes.c_int,
                                 _D, P(ctypes.c_int)]
    L.sph_batch_adapt.restype = ctypes.c_int
    L.sph_batch_adapt.argtypes = [ctypes.c_void_p, P(ctypes.c_void_p), ctypes.c_int,
                                  P(AdaptStats), P(ctypes.c_int)]
    L.sph_batch_launches.restype = ctypes.c_longlong
    L.sph_batch_launches.argtypes = [ctypes.c_void_p]
    L.sph_batch_graph_steps.restype = ctypes.c_longlong
    L.sph_batch_graph_steps.argtypes = [ctypes.c_void_p]
    L.sph_batch_set_graphs.restype = ctypes.c_int
    L.sph_batch_set_graphs.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.sph_force_coefficients.restype = ctypes.c_int
    L.sph_force_coefficients.argtypes = [ctx, ctypes.c_double, ctypes.c_double, _D]
    L.sph_debug_failures.restype = ctypes.c_ulonglong
    L.sph_debug_failures.argtypes = []
    L.sph_debug_build.restype = ctypes.c_int
    L.sph_debug_build.argtypes = []
    L.sph_probe_fma.restype = ctypes.c_int
    L.sph_probe_fma.argtypes = [ctypes.c_int, ctypes.c_void_p, _D, P(ctypes.c_int)]
    _lib = L
    return L


def _tune_dict(t: Tune) -> dict:
    out = {k: getattr(t, k) for k in ("cell_scale", "walk", "team_a", "team_b",
                                      "walls", "no_graphs")}
    for k in ("ms_cell", "ms_walk", "ms_team_a", "ms_team_b", "ms_walls"):
        out[k] = list(getattr(t, k))
    return out


def probe_fma(fp64: bool = False, stream: int = 0) -> tuple:
    """sph_probe_fma: measured FMA rate (FLOP/s) of the device and its SM
    count."""
    L = lib()
    fl = ctypes.c_double(0.0)
    sms = ctypes.c_int(0)
    st = L.sph_probe_fma(1 if fp64 else 0, ctypes.c_void_p(stream),
                         ctypes.byref(fl), ctypes.byref(sms))
    if st != SPH_OK:
        raise SphError(st, "sph_probe_fma failed")
    return fl.value, sms.value


def cell_sort_noalloc(params: Params, n: int, x_ptr: int, y_ptr: int,
                      h_ptr: int, key_ptr: int, perm_ptr: int,
                      stream: int = 0) -> int:
    """sph_cell_sort_noalloc on caller-owned device pointers; returns the
    status code."""
    v = ctypes.c_void_p
    return lib().sph_cell_sort_noalloc(ctypes.byref(params), int(n),
                                       v(x_ptr), v(y_ptr), v(h_ptr),
                                       v(key_ptr), v(perm_ptr), v(stream))


def debug_failures() -> int:
    """sph_debug_failures: bounds-check failures counted by a debug build
    since the last call (always 0 in a release build)."""
    return int(lib().sph_debug_failures())


def debug_build() -> bool:
    """sph_debug_build: whether the loaded library has the checks."""
    return bool(lib().sph_debug_build())


def last_error() -> str:
    """sph_last_error(NULL): the reason of the calling thread's last failed
    call made without a context (sph_create, sph_cell_sort_noalloc)."""
    return lib().sph_last_error(None).decode()


def declared_functions():
    """Names of the functions include/sph.h declares."""
    txt = open(os.path.join(_build.INCLUDE, "sph.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", txt)))


def make_params(d: dict, precision: int = SPH_FP64, capacity: int = 0,
                **over) -> Params:
    """sph_params from a workload's parameter dict (unknown keys ignored)."""
    P = Params()
    lib().sph_default_params(ctypes.byref(P))
    d = dict(d)
    d.update(over)
    for k, v in d.items():
        if k in ("lo", "hi"):
            getattr(P, k)[:] = [float(a) for a in v]
        elif k == "periodic":
            P.periodic[:] = [int(a) for a in v]
        elif k in dict(Params._fields_):
            t = dict(Params._fields_)[k]
            setattr(P, k, int(v) if t in (ctypes.c_int, ctypes.c_longlong)
                    else float(v))
    P.precision = int(precision)
    P.capacity = int(capacity)
    return P


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Simulation:
    """One sph_ctx.  ``stream`` is a cudaStream_t handle (int), 0 for the
    legacy default stream."""

    def __init__(self, params: Params, stream: int = 0):
        self._L = lib()
        self._ctx = ctypes.c_void_p()
        st = self._L.sph_create(ctypes.byref(params),
                                ctypes.c_void_p(int(stream)),
                                ctypes.byref(self._ctx))
        if st != SPH_OK:
            raise SphError(st, self._L.sph_last_error(None).decode())
        self.params = params
        self._keep = []

    def _check(self, st):
        if st != SPH_OK:
            raise SphError(st, self._L.sph_last_error(self._ctx).decode())

    def load(self, particles: dict, kind: int = SPH_FLUID):
        n = len(particles["x"])
        src = Particles()
        keep = []
        for k in ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax",
                  "ds"):
            if k in particles and particles[k] is not None:
                a = _f64(particles[k])
                keep.append(a)
                setattr(src, k, a.ctypes.data_as(_D))
        if "id" in particles and particles["id"] is not None:
            a = np.ascontiguousarray(particles["id"], dtype=np.int64)
            keep.append(a)
            src.id = a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        self._check(self._L.sph_load_particles(self._ctx, int(kind), n,
                                               ctypes.byref(src)))

    def load_raw(self, kind: int, n: int, src: Particles):
        """sph_load_particles with a caller-built Particles block (pinned
        host buffers for end-to-end timing)."""
        self._check(self._L.sph_load_particles(self._ctx, int(kind), int(n),
                                               ctypes.byref(src)))

    def rhs(self):
        self._check(self._L.sph_rhs(self._ctx))

    def step(self, nsteps: int = 1, want_time: bool = True):
        t = ctypes.c_double(0.0)
        self._check(self._L.sph_step(self._ctx, int(nsteps),
                                     ctypes.byref(t) if want_time else None))
        return t.value if want_time else None

    def adapt(self) -> dict:
        z = AdaptStats()
        self._check(self._L.sph_adapt(self._ctx, ctypes.byref(z)))
        return {k: getattr(z, k) for k, _ in AdaptStats._fields_}

    def background(self, iterations: int = 0) -> dict:
        """sph_background: ``iterations`` construction iterations (0: the
        paper's count for the initial construction)."""
        z = BgStats()
        self._check(self._L.sph_background(self._ctx, int(iterations),
                                           ctypes.byref(z)))
        return {k: getattr(z, k) for k, _ in BgStats._fields_}

    def autotune(self) -> dict:
        """sph_autotune: time the launch configurations on the loaded set
        and keep the fastest; returns the choices and the times."""
        t = Tune()
        self._check(self._L.sph_autotune(self._ctx, ctypes.byref(t)))
        return _tune_dict(t)

    def set_tuning(self, cell_scale: float = 1.0, walk: int = 0,
                   team_a: int = 0, team_b: int = 0, graphs: bool = True,
                   walls: int = 0):
        """sph_set_tuning (0: the size rule; graphs False: sph_step launch
        by launch; walls 1 cell walk, 2 wall lists)."""
        t = Tune()
        t.cell_scale, t.walk, t.team_a, t.team_b = cell_scale, walk, team_a, team_b
        t.walls = walls
        t.no_graphs = 0 if graphs else 1
        self._check(self._L.sph_set_tuning(self._ctx, ctypes.byref(t)))

    def forces(self, per_wall: bool = False) -> dict:
        """sph_forces: force on the wall particles at the current state,
        {"fp": (x, y) pressure part, "fv": (x, y) viscous part} and, with
        per_wall, "per_wall": (n_walls, 4) in load order."""
        tot = np.zeros(4)
        nw = self.info()["n_wall"]
        pw = np.zeros((max(nw, 1), 4)) if per_wall else None
        self._check(self._L.sph_forces(
            self._ctx, pw.ctypes.data if per_wall else None,
            tot.ctypes.data_as(_D)))
        out = {"fp": tot[:2].copy(), "fv": tot[2:].copy()}
        if per_wall:
            out["per_wall"] = pw[:nw]
        return out

    def coefficients(self, U: float, L: float) -> dict:
        """sph_force_coefficients: pressure drag, skin-friction drag and lift
        coefficients (Eq. cdcl) at the current state."""
        out = (ctypes.c_double * 3)()
        self._check(self._L.sph_force_coefficients(self._ctx, float(U), float(L), out))
        return {"cd_p": out[0], "cd_sf": out[1], "cl": out[2]}

    def read_background(self) -> dict:
        """The background set (x, y, h, m, ds, id) in the library's order."""
        return {k: self.read("bg_" + k) for k in ("x", "y", "h", "m", "ds", "id")}

    def read(self, field: str, by_id: bool = False) -> np.ndarray:
        """sph_read of one field; by_id: rows in ascending id order
        (SPH_READ_BY_ID) instead of the library's current order."""
        f = FIELD[field] | (SPH_READ_BY_ID if by_id else 0)
        dt = _FIELD_DTYPE.get(field, np.float64)
        n = ctypes.c_longlong(0)
        st = self._L.sph_read(self._ctx, f, None, 0, ctypes.byref(n))
        if st not in (SPH_OK, SPH_ECAPACITY):
            self._check(st)
        out = np.zeros(max(n.value, 1), dtype=dt)
        self._check(self._L.sph_read(self._ctx, f,
                                     out.ctypes.data_as(ctypes.c_void_p),
                                     out.size, ctypes.byref(n)))
        return out[:n.value]

    def read_into(self, field: str, out: np.ndarray) -> int:
        n = ctypes.c_longlong(0)
        self._check(self._L.sph_read(self._ctx, FIELD[field],
                                     out.ctypes.data_as(ctypes.c_void_p),
                                     out.size, ctypes.byref(n)))
        return n.value

    def info(self) -> dict:
        i = Info()
        self._check(self._L.sph_get_info(self._ctx, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def set_timing(self, on: bool):
        self._check(self._L.sph_set_timing(self._ctx, 1 if on else 0))

    def kernel_time(self, family: int, reset: bool = False):
        ms = ctypes.c_double(0)
        cnt = ctypes.c_longlong(0)
        self._check(self._L.sph_kernel_time(self._ctx, family,
                                            ctypes.byref(ms),
                                            ctypes.byref(cnt), int(reset)))
        return ms.value, cnt.value

    def close(self):
        if self._ctx:
            self._L.sph_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Several simulations stepped together (sph_batch_*): each context's
    neighbour build on its own stream, every per-particle phase as one
    persistent launch over all of them on ``stream``."""

    def __init__(self, max_instances: int, stream: int = 0):
        self._L = lib()
        self._b = ctypes.c_void_p()
        st = self._L.sph_batch_create(int(max_instances), ctypes.c_void_p(int(stream)),
                                      ctypes.byref(self._b))
        if st != SPH_OK:
            raise SphError(st, "sph_batch_create failed")
        self.max_instances = int(max_instances)

    def step(self, sims, want_time: bool = False):
        """One PEC step of every Simulation in ``sims``; with want_time the
        simulated times (one synchronisation)."""
        k = len(sims)
        arr = (ctypes.c_void_p * max(k, 1))(*[s._ctx.value for s in sims])
        t = np.zeros(max(k, 1), np.float64)
        failed = ctypes.c_int(-1)
        st = self._L.sph_batch_step(self._b, arr, k,
                                    t.ctypes.data_as(_D) if want_time else None,
                                    ctypes.byref(failed))
        if st != SPH_OK:
            q = failed.value
            msg = (self._L.sph_last_error(sims[q]._ctx).decode()
                   if 0 <= q < k else "sph_batch_step failed")
            raise SphError(st, msg)
        return t[:k] if want_time else None

    def adapt(self, sims, errors: str = "raise"):
        """One sph_adapt of every Simulation in ``sims``, in lockstep
        (sph_batch_adapt): a list of stats dicts.  errors="raise" raises the
        first failed context's error; errors="return" puts (status,
        message) in a failed context's place instead."""
        k = len(sims)
        arr = (ctypes.c_void_p * max(k, 1))(*[s._ctx.value for s in sims])
        z = (AdaptStats * max(k, 1))()
        stat = (ctypes.c_int * max(k, 1))()
        st = self._L.sph_batch_adapt(self._b, arr, k, z, stat)
        if st == SPH_EINVAL and all(v == 0 for v in stat[:k]):
            raise SphError(st, "sph_batch_adapt: invalid arguments")
        out = []
        for q in range(k):
            if stat[q] != SPH_OK:
                msg = self._L.sph_last_error(sims[q]._ctx).decode()
                if errors == "raise":
                    raise SphError(stat[q], msg)
                out.append((stat[q], msg))
            else:
                out.append({f: getattr(z[q], f) for f, _ in AdaptStats._fields_})
        return out

    @property
    def launches(self) -> int:
        return int(self._L.sph_batch_launches(self._b))

    @property
    def graph_steps(self) -> int:
        return int(self._L.sph_batch_graph_steps(self._b))

    def set_graphs(self, enable: bool):
        if self._L.sph_batch_set_graphs(self._b, int(bool(enable))) != SPH_OK:
            raise SphError(SPH_EINVAL, "sph_batch_set_graphs failed")

    def close(self):
        if self._b:
            self._L.sph_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
