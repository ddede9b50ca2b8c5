"""Plain FP64 CPU oracle for the adaptive-resolution WCSPH method of
Muta & Ramachandran (arXiv 2107.01276).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  It
shares no code with the CUDA library (``paper_2107_01276_gb300``) and never
imports it; the CUDA library never imports this.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, FMA contraction
off).  This module only compiles it with gcc, loads it with ctypes and
marshals numpy arrays.  Functions whose parity is not pinned by a test
against the paper or mathematics say so in their docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsph_oracle.so")
_SRC = [os.path.join(_HERE, "sph_oracle.c")]
_HDR = os.path.join(_HERE, "sph_oracle.h")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no GPU involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
        ("periodic", ctypes.c_int * 2),
        ("rho0", ctypes.c_double), ("cs", ctypes.c_double),
        ("nu", ctypes.c_double), ("U_ref", ctypes.c_double),
        ("hdx", ctypes.c_double), ("alpha_e", ctypes.c_double),
        ("split_alpha", ctypes.c_double), ("split_eps", ctypes.c_double),
        ("pavg_mode", ctypes.c_int), ("edac_diff_denominator", ctypes.c_int),
        ("edac_rho_factor", ctypes.c_int), ("merge_iters", ctypes.c_int),
        ("shift_iters", ctypes.c_int),
    ]


class _State(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("cap", ctypes.c_int)] + [
        (k, ctypes.POINTER(ctypes.c_double))
        for k in ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax")
    ] + [("id", ctypes.POINTER(ctypes.c_longlong))]


_RHS_D = ("rho", "beta", "pavg", "drx", "dry", "dpdt", "dudt", "dvdt")
_RHS_S = tuple("s_" + k for k in ("rho", "beta", "pavg", "drx", "dry",
                                  "dpdt", "dudt", "dvdt"))


class _RhsOut(ctypes.Structure):
    _fields_ = [(k, ctypes.POINTER(ctypes.c_double)) for k in _RHS_D] + [
        ("nnb", ctypes.POINTER(ctypes.c_int))] + [
        (k, ctypes.POINTER(ctypes.c_double)) for k in _RHS_S]


class _AdaptStats(ctypes.Structure):
    _fields_ = [("n_before", ctypes.c_longlong), ("n_split", ctypes.c_longlong),
                ("n_merged", ctypes.c_longlong), ("n_after", ctypes.c_longlong),
                ("mass_before", ctypes.c_double),
                ("mass_after", ctypes.c_double)]


class _BgSet(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("cap", ctypes.c_int)] + [
        (k, ctypes.POINTER(ctypes.c_double)) for k in ("x", "y", "h", "m", "ds")
    ] + [("id", ctypes.POINTER(ctypes.c_longlong))]


class BgParams(ctypes.Structure):
    _fields_ = [("ds_min", ctypes.c_double), ("ds_max", ctypes.c_double),
                ("Cr", ctypes.c_double), ("Nr", ctypes.c_double),
                ("smooth_iters", ctypes.c_int), ("vort_k", ctypes.c_double)]


class _BgStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in
                ("n_before", "n_marked", "n_vort", "n_split", "n_after")]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_P = ctypes.POINTER(Params)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_W.restype = ctypes.c_double
            L.orc_W.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_dWdr.restype = ctypes.c_double
            L.orc_dWdr.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_is_neighbor.restype = ctypes.c_int
            L.orc_is_neighbor.argtypes = [_P] + [ctypes.c_double] * 6
            for f in (L.orc_neighbors_brute, L.orc_neighbors_grid):
                f.restype = ctypes.c_longlong
                f.argtypes = [_P, ctypes.c_int, _D, _D, _D, _I, _I,
                              ctypes.c_longlong]
            L.orc_neighbors_cross.restype = ctypes.c_longlong
            L.orc_neighbors_cross.argtypes = [_P, ctypes.c_int, _D, _D, _D,
                                              ctypes.c_int, _D, _D, _D, _I,
                                              _I, ctypes.c_longlong]
            L.orc_max_level.restype = ctypes.c_int
            L.orc_max_level.argtypes = [_P, ctypes.c_double]
            L.orc_cell_keys.restype = None
            L.orc_cell_keys.argtypes = [_P, ctypes.c_double, ctypes.c_int,
                                        _D, _D, _D, _U64, _I]
            L.orc_pass_a.restype = ctypes.c_int
            L.orc_pass_a.argtypes = [_P, ctypes.c_int, _D, _D, _D, _D, _D,
                                     _I, _I, ctypes.POINTER(_RhsOut)]
            L.orc_pass_b.restype = None
            L.orc_pass_b.argtypes = [_P, ctypes.c_double, ctypes.c_int, _D,
                                     _D, _D, _D, _D, _D, _D, _I, _I,
                                     ctypes.POINTER(_RhsOut)]
            L.orc_dt.restype = ctypes.c_double
            L.orc_dt.argtypes = [_P, ctypes.c_int, _D]
            L.orc_rhs.restype = ctypes.c_int
            L.orc_rhs.argtypes = [_P, ctypes.c_double,
                                  ctypes.POINTER(_State),
                                  ctypes.POINTER(_RhsOut)]
            L.orc_step.restype = ctypes.c_int
            L.orc_step.argtypes = [_P, ctypes.POINTER(_State), ctypes.c_int,
                                   _D]
            for f in (L.orc_pec_predict, L.orc_pec_correct):
                f.restype = None
                f.argtypes = [_P, ctypes.c_double, ctypes.c_int] + [_D] * 15
            L.orc_bg_resolution.restype = None
            L.orc_bg_resolution.argtypes = [_P, ctypes.POINTER(_State),
                                            ctypes.c_int, _D, _D, _D, _D]
            L.orc_split.restype = ctypes.c_int
            L.orc_split.argtypes = [_P, ctypes.POINTER(_State),
                                    ctypes.POINTER(ctypes.c_longlong)]
            L.orc_merge_round.restype = ctypes.c_int
            L.orc_merge_round.argtypes = [_P, ctypes.POINTER(_State)]
            L.orc_shift_compute.restype = None
            L.orc_shift_compute.argtypes = [_P, ctypes.POINTER(_State)] + \
                [_D] * 9
            L.orc_shift_round.restype = None
            L.orc_shift_round.argtypes = [_P, ctypes.POINTER(_State)]
            L.orc_h_update.restype = None
            L.orc_h_update.argtypes = [_P, ctypes.POINTER(_State)]
            L.orc_adapt.restype = ctypes.c_int
            L.orc_adapt.argtypes = [_P, ctypes.POINTER(_State), ctypes.c_int,
                                    _D, _D, _D, _D,
                                    ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(_AdaptStats)]
            L.orc_set_walls.restype = None
            L.orc_set_walls.argtypes = [ctypes.c_int] + [_D] * 6
            L.orc_wall_bc.restype = None
            L.orc_wall_bc.argtypes = [_P, ctypes.POINTER(_State), _D, _D, _D]
            L.orc_wall_bc_store.restype = None
            L.orc_wall_bc_store.argtypes = [_P, ctypes.POINTER(_State)]
            L.orc_forces.restype = None
            L.orc_forces.argtypes = [_P, ctypes.POINTER(_State), _D, ctypes.c_void_p]
            L.orc_record_wall_terms.restype = None
            L.orc_record_wall_terms.argtypes = [ctypes.c_void_p]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_num_threads.argtypes = []
            L.orc_set_num_threads.restype = None
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_neighbors_classes.restype = ctypes.c_longlong
            L.orc_neighbors_classes.argtypes = [_P, ctypes.c_int, _D, _D, _D,
                                                _I, _I, ctypes.c_longlong]
            _BG = ctypes.POINTER(_BgSet)
            _BP = ctypes.POINTER(BgParams)
            _LL = ctypes.POINTER(ctypes.c_longlong)
            _U8 = ctypes.POINTER(ctypes.c_uint8)
            L.orc_bg_iterations.restype = ctypes.c_int
            L.orc_bg_iterations.argtypes = [_BP]
            L.orc_vorticity.restype = None
            L.orc_vorticity.argtypes = [_P, ctypes.POINTER(_State), _D]
            L.orc_bg_mark.restype = ctypes.c_int
            L.orc_bg_mark.argtypes = [_P, _BP, _BG, ctypes.c_int, _D, _D, _D,
                                      ctypes.c_int, _D, _D, _D, _D, _U8]
            L.orc_bg_size.restype = None
            L.orc_bg_size.argtypes = [_P, _BP, _BG, _U8]
            L.orc_bg_split.restype = ctypes.c_int
            L.orc_bg_split.argtypes = [_P, _BG, _LL]
            L.orc_bg_hsmooth.restype = None
            L.orc_bg_hsmooth.argtypes = [_P, _BP, _BG]
            L.orc_bg_shift.restype = None
            L.orc_bg_shift.argtypes = [_P, _BG]
            L.orc_bg_iteration.restype = ctypes.c_int
            L.orc_bg_iteration.argtypes = [_P, _BP, _BG, _LL, ctypes.c_int,
                                           _D, _D, _D, ctypes.c_int, _D, _D,
                                           _D, _D,
                                           ctypes.POINTER(_BgStats)]
            _lib = L
    return _lib


PARAM_DEFAULTS = dict(
    lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(0, 0), rho0=1.0, cs=10.0,
    nu=0.0, U_ref=1.0, hdx=1.0, alpha_e=1.5, split_alpha=0.9, split_eps=0.4,
    pavg_mode=0, edac_diff_denominator=1, edac_rho_factor=1, merge_iters=3,
    shift_iters=3)


def params(**kw) -> Params:
    """Build the oracle parameter block; unspecified fields take the
    paper's values (alpha_e 1.5, split alpha 0.9, epsilon 0.4, three merge
    and shift rounds) and the default readings."""
    d = dict(PARAM_DEFAULTS)
    for k, v in kw.items():
        if k in d:
            d[k] = v
    P = Params()
    P.lo[:] = [float(v) for v in d["lo"]]
    P.hi[:] = [float(v) for v in d["hi"]]
    P.periodic[:] = [int(v) for v in d["periodic"]]
    for k in ("rho0", "cs", "nu", "U_ref", "hdx", "alpha_e", "split_alpha",
              "split_eps"):
        setattr(P, k, float(d[k]))
    for k in ("pavg_mode", "edac_diff_denominator", "edac_rho_factor",
              "merge_iters", "shift_iters"):
        setattr(P, k, int(d[k]))
    return P


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (timing only: the results do
    not depend on the count)."""
    lib().orc_set_num_threads(int(n))


def W(r, h):
    """Quintic spline W(r, h) (section 2, Eq. kernel), elementwise."""
    L = lib()
    r, h = np.broadcast_arrays(np.asarray(r, float), np.asarray(h, float))
    return np.array([L.orc_W(a, b) for a, b in zip(r.ravel(), h.ravel())]
                    ).reshape(r.shape)


def dWdr(r, h):
    L = lib()
    r, h = np.broadcast_arrays(np.asarray(r, float), np.asarray(h, float))
    return np.array([L.orc_dWdr(a, b) for a, b in zip(r.ravel(), h.ravel())]
                    ).reshape(r.shape)


def is_neighbor(P, xi, yi, hi, xj, yj, hj) -> bool:
    return bool(lib().orc_is_neighbor(ctypes.byref(P), xi, yi, hi, xj, yj,
                                      hj))


def neighbors(P, x, y, h, method: str = "grid"):
    """CSR (off, nbr) of N(i) = {j : r_ij < 3 max(h_i, h_j)}, ascending j."""
    x, y, h = _f64(x), _f64(y), _f64(h)
    n = len(x)
    f = lib().orc_neighbors_grid if method == "grid" else \
        lib().orc_neighbors_brute
    off = np.zeros(n + 1, np.int32)
    cap = max(64, 48 * n)
    while True:
        nbr = np.zeros(cap, np.int32)
        tot = f(ctypes.byref(P), n, _d(x), _d(y), _d(h), _i(off), _i(nbr),
                cap)
        if tot <= cap:
            return off, nbr[:tot].copy()
        cap = int(tot)


def neighbors_cross(P, xa, ya, ha, xb, yb, hb):
    xa, ya, ha, xb, yb, hb = map(_f64, (xa, ya, ha, xb, yb, hb))
    na, nb = len(xa), len(xb)
    off = np.zeros(na + 1, np.int32)
    cap = max(64, 48 * na)
    while True:
        nbr = np.zeros(cap, np.int32)
        tot = lib().orc_neighbors_cross(ctypes.byref(P), na, _d(xa), _d(ya),
                                        _d(ha), nb, _d(xb), _d(yb), _d(hb),
                                        _i(off), _i(nbr), cap)
        if tot <= cap:
            return off, nbr[:tot].copy()
        cap = int(tot)


def max_level(P, c0: float) -> int:
    return int(lib().orc_max_level(ctypes.byref(P), float(c0)))


def cell_keys(P, c0, x, y, h):
    """Multi-level cell key and level of every particle (definition in
    sph_oracle.c).  Returns (key uint64[n], level int32[n])."""
    x, y, h = _f64(x), _f64(y), _f64(h)
    n = len(x)
    key = np.zeros(n, np.uint64)
    lev = np.zeros(n, np.int32)
    lib().orc_cell_keys(ctypes.byref(P), float(c0), n, _d(x), _d(y), _d(h),
                        key.ctypes.data_as(_U64), _i(lev))
    return key, lev


def _rhs_out(n):
    arrs = {k: np.zeros(max(n, 1)) for k in _RHS_D + _RHS_S}
    arrs["nnb"] = np.zeros(max(n, 1), np.int32)
    o = _RhsOut()
    for k in _RHS_D + _RHS_S:
        setattr(o, k, _d(arrs[k]))
    o.nnb = _i(arrs["nnb"])
    return o, arrs


def pass_a(P, x, y, h, m, p, off, nbr):
    x, y, h, m, p = map(_f64, (x, y, h, m, p))
    n = len(x)
    o, arrs = _rhs_out(n)
    off = np.ascontiguousarray(off, np.int32)
    nbr = np.ascontiguousarray(nbr, np.int32)
    lib().orc_pass_a(ctypes.byref(P), n, _d(x), _d(y), _d(h), _d(m), _d(p),
                     _i(off), _i(nbr), ctypes.byref(o))
    return {k: v[:n] for k, v in arrs.items()}


def pass_b(P, dt, x, y, h, m, p, u, v, off, nbr, a):
    """Pass B with pass-A results ``a`` (rho, beta, pavg, drx, dry) given;
    the caller may prescribe them (used by the pins)."""
    x, y, h, m, p, u, v = map(_f64, (x, y, h, m, p, u, v))
    n = len(x)
    o, arrs = _rhs_out(n)
    for k in ("rho", "beta", "pavg", "drx", "dry"):
        arrs[k][:n] = a[k]
    off = np.ascontiguousarray(off, np.int32)
    nbr = np.ascontiguousarray(nbr, np.int32)
    lib().orc_pass_b(ctypes.byref(P), float(dt), n, _d(x), _d(y), _d(h),
                     _d(m), _d(p), _d(u), _d(v), _i(off), _i(nbr),
                     ctypes.byref(o))
    return {k: v[:n] for k, v in arrs.items()}


def dt(P, h) -> float:
    h = _f64(h)
    return float(lib().orc_dt(ctypes.byref(P), len(h), _d(h)))


STATE_FIELDS = ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax")


def make_state(fields: dict, cap: int | None = None) -> dict:
    """Copy a particle dict into capacity-sized FP64 arrays owned here."""
    n = len(fields["x"])
    cap = max(n, cap or n, 1)
    st = {"n": n, "cap": cap}
    for k in STATE_FIELDS:
        a = np.zeros(cap)
        if k in fields:
            a[:n] = fields[k]
        st[k] = a
    ida = np.zeros(cap, np.int64)
    ida[:n] = fields.get("id", np.arange(n))
    st["id"] = ida
    return st


def _cstate(st):
    s = _State()
    s.n, s.cap = st["n"], st["cap"]
    for k in STATE_FIELDS:
        setattr(s, k, _d(st[k]))
    s.id = st["id"].ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    return s


def rhs(P, dt_, st):
    """Neighbour search + pass A + pass B at the state ``st``."""
    n = st["n"]
    o, arrs = _rhs_out(n)
    s = _cstate(st)
    lib().orc_rhs(ctypes.byref(P), float(dt_), ctypes.byref(s),
                  ctypes.byref(o))
    return {k: v[:n].copy() for k, v in arrs.items()}


def step(P, st, nsteps: int, t: float = 0.0) -> float:
    """Advance ``st`` in place by nsteps PEC steps; returns the new time."""
    s = _cstate(st)
    tt = ctypes.c_double(t)
    lib().orc_step(ctypes.byref(P), ctypes.byref(s), int(nsteps),
                   ctypes.byref(tt))
    st["n"] = s.n
    return tt.value


def pec_stage(P, which, dt_, x0, y0, u0, v0, p0, dudt, dvdt, dpdt, drx,
              dry):
    arrs = list(map(_f64, (x0, y0, u0, v0, p0, dudt, dvdt, dpdt, drx, dry)))
    n = len(arrs[0])
    out = [np.zeros(n) for _ in range(5)]
    f = lib().orc_pec_predict if which == "predict" else \
        lib().orc_pec_correct
    f(ctypes.byref(P), float(dt_), n, *[_d(a) for a in arrs],
      *[_d(a) for a in out])
    return dict(zip(("x", "y", "u", "v", "p"), out))


# ---------------------------------------------------------- adaptation --
def _bg(bg):
    if bg is None:
        z = np.zeros(1)
        return 0, z, z, z, z
    arrs = [_f64(bg[k]) for k in ("x", "y", "h", "ds")]
    return len(arrs[0]), arrs[0], arrs[1], arrs[2], arrs[3]


def bg_resolution(P, st, bg):
    """Fluid m_min, m_max from background particles (dict x, y, h, ds)."""
    nb, bx, by, bh, bd = _bg(bg)
    s = _cstate(st)
    lib().orc_bg_resolution(ctypes.byref(P), ctypes.byref(s), nb, _d(bx),
                            _d(by), _d(bh), _d(bd))


def split(P, st, next_id):
    """One split pass; returns (parents split or -1, new next_id)."""
    s = _cstate(st)
    nid = ctypes.c_longlong(int(next_id))
    r = lib().orc_split(ctypes.byref(P), ctypes.byref(s), ctypes.byref(nid))
    st["n"] = s.n
    return r, nid.value


def merge_round(P, st):
    s = _cstate(st)
    r = lib().orc_merge_round(ctypes.byref(P), ctypes.byref(s))
    st["n"] = s.n
    return r


def shift_compute(P, st):
    n = st["n"]
    out = {k: np.zeros(max(n, 1)) for k in ("rho", "drx", "dry", "gux",
                                             "guy", "gvx", "gvy", "gpx",
                                             "gpy")}
    s = _cstate(st)
    lib().orc_shift_compute(ctypes.byref(P), ctypes.byref(s),
                            *[_d(out[k]) for k in ("rho", "drx", "dry", "gux",
                                                   "guy", "gvx", "gvy", "gpx",
                                                   "gpy")])
    return {k: v[:n] for k, v in out.items()}


def shift_round(P, st):
    s = _cstate(st)
    lib().orc_shift_round(ctypes.byref(P), ctypes.byref(s))


def h_update(P, st):
    s = _cstate(st)
    lib().orc_h_update(ctypes.byref(P), ctypes.byref(s))


def adapt(P, st, bg=None, next_id=None):
    """One adaptation (background resolution, split, merge rounds, shift
    rounds, h update) in place; returns (status, stats dict, next_id)."""
    nb, bx, by, bh, bd = _bg(bg)
    if next_id is None:
        next_id = int(st["id"][:st["n"]].max()) + 1 if st["n"] else 0
    s = _cstate(st)
    nid = ctypes.c_longlong(int(next_id))
    z = _AdaptStats()
    r = lib().orc_adapt(ctypes.byref(P), ctypes.byref(s), nb, _d(bx), _d(by),
                        _d(bh), _d(bd), ctypes.byref(nid), ctypes.byref(z))
    st["n"] = s.n
    return r, {k: getattr(z, k) for k, _ in _AdaptStats._fields_}, nid.value


# --------------------------------------------------------------- walls --
def set_walls(walls):
    """Register dummy wall particles (dict x, y, h, m, optional u, v) for
    rhs/step/adapt; None clears them."""
    if walls is None or len(walls["x"]) == 0:
        lib().orc_set_walls(0, None, None, None, None, None, None)
        return
    n = len(walls["x"])
    arrs = [_f64(walls[k]) for k in ("x", "y", "h", "m")]
    arrs.append(_f64(walls.get("u", np.zeros(n))))
    arrs.append(_f64(walls.get("v", np.zeros(n))))
    lib().orc_set_walls(n, *[_d(a) for a in arrs])


def wall_bc_store(P, st):
    """Evaluate the wall condition at the state and keep it for the
    registered walls (before calling pass_a / pass_b with walls)."""
    s = _cstate(st)
    lib().orc_wall_bc_store(ctypes.byref(P), ctypes.byref(s))


def wall_bc(P, st, nw):
    """Wall pressure and extrapolated velocity of the registered walls."""
    out = [np.zeros(max(nw, 1)) for _ in range(3)]
    s = _cstate(st)
    lib().orc_wall_bc(ctypes.byref(P), ctypes.byref(s), *[_d(a) for a in out])
    return {"p": out[0][:nw], "ugx": out[1][:nw], "ugy": out[2][:nw]}


def forces(P, st, nw: int = 0):
    """Force on the registered walls at the state (section "Force
    computation", Eq. force-sph): dict fp (pressure), fv (viscous), each
    an (x, y) array, and with nw > 0 (the wall count) "per_wall", (nw, 4)."""
    out = np.zeros(4)
    pw = np.zeros((nw, 4)) if nw > 0 else None
    s = _cstate(st)
    lib().orc_forces(ctypes.byref(P), ctypes.byref(s), _d(out),
                     pw.ctypes.data if pw is not None else None)
    r = {"fp": out[:2].copy(), "fv": out[2:].copy()}
    if pw is not None:
        r["per_wall"] = pw
    return r


def coefficients(f, rho0, U, L):
    """Eq. cdcl: pressure drag, skin-friction drag and lift coefficients
    from a forces() dict, with the dynamic pressure rho0 U^2 / 2 and the
    characteristic length L."""
    q = 0.5 * rho0 * U * U * L
    return {"cd_p": f["fp"][0] / q, "cd_sf": f["fv"][0] / q,
            "cl": f["fp"][1] / q}


def rhs_wall_terms(P, dt_, st):
    """One right-hand side with each fluid particle's wall terms of its
    momentum rate: (out dict of rhs, array n x 4 of pressure x, y and
    viscous x, y wall terms)."""
    n = st["n"]
    acc = np.zeros((max(n, 1), 4))
    lib().orc_record_wall_terms(acc.ctypes.data)
    try:
        out = rhs(P, dt_, st)
    finally:
        lib().orc_record_wall_terms(None)
    return out, acc[:n]


# ---------------------------------------------------------- background --
BG_FIELDS = ("x", "y", "h", "m", "ds")


def bg_params(ds_min, ds_max, Cr=1.08, Nr=48.0, smooth_iters=3, vort_k=0.0):
    """Background construction parameters (section 3.3; N_r = 48 and three
    smoothing repetitions are the paper's)."""
    B = BgParams()
    B.ds_min, B.ds_max, B.Cr, B.Nr = float(ds_min), float(ds_max), float(Cr), \
        float(Nr)
    B.smooth_iters, B.vort_k = int(smooth_iters), float(vort_k)
    return B


def make_bgset(fields: dict, cap: int | None = None) -> dict:
    """Background set arrays (x, y, h, m, ds, id) with capacity ``cap``."""
    n = len(fields["x"])
    cap = max(n, cap or n, 1)
    b = {"n": n, "cap": cap}
    for k in BG_FIELDS:
        a = np.zeros(cap)
        a[:n] = fields[k]
        b[k] = a
    ida = np.zeros(cap, np.int64)
    ida[:n] = fields.get("id", np.arange(n))
    b["id"] = ida
    return b


def _cbg(b):
    s = _BgSet()
    s.n, s.cap = b["n"], b["cap"]
    for k in BG_FIELDS:
        setattr(s, k, _d(b[k]))
    s.id = b["id"].ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    return s


def _sync_bg(b, s):
    b["n"] = s.n


def neighbors_classes(P, x, y, h):
    """Same sets as ``neighbors`` by the h-class bucket search."""
    x, y, h = _f64(x), _f64(y), _f64(h)
    n = len(x)
    off = np.zeros(n + 1, np.int32)
    cap = max(64, 48 * n)
    while True:
        nbr = np.zeros(cap, np.int32)
        tot = lib().orc_neighbors_classes(ctypes.byref(P), n, _d(x), _d(y),
                                          _d(h), _i(off), _i(nbr), cap)
        if tot <= cap:
            return off, nbr[:tot].copy()
        cap = int(tot)


def bg_iterations(B) -> int:
    return int(lib().orc_bg_iterations(ctypes.byref(B)))


def vorticity(P, st):
    """omega_i of the fluid state (gradient operator of the Taylor
    correction)."""
    n = st["n"]
    out = np.zeros(max(n, 1))
    s = _cstate(st)
    lib().orc_vorticity(ctypes.byref(P), ctypes.byref(s), _d(out))
    return out[:n]


def _solid_fluid(solid, fluid):
    z = np.zeros(1)
    if solid is None or len(solid["x"]) == 0:
        sw = (0, z, z, z)
    else:
        sw = (len(solid["x"]),) + tuple(_f64(solid[k]) for k in ("x", "y", "h"))
    if fluid is None or len(fluid["x"]) == 0:
        fl = (0, z, z, z, None)
    else:
        fl = (len(fluid["x"]),) + tuple(_f64(fluid[k]) for k in ("x", "y", "h")) \
            + (_f64(fluid["phi"]),)
    return sw, fl


def bg_mark(P, B, b, solid, fluid=None):
    """Step 1 in place; returns the mark array (0, 1 solid, 2 vorticity).
    ``fluid``: dict x, y, h, phi (= |omega|) or None."""
    (nw, wx, wy, wh), (nf, fx, fy, fh, phi) = _solid_fluid(solid, fluid)
    mark = np.zeros(max(b["n"], 1), np.uint8)
    s = _cbg(b)
    lib().orc_bg_mark(ctypes.byref(P), ctypes.byref(B), ctypes.byref(s), nw,
                      _d(wx), _d(wy), _d(wh), nf, _d(fx), _d(fy), _d(fh),
                      _d(phi) if phi is not None else None,
                      mark.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return mark[:b["n"]]


def bg_size(P, B, b, mark):
    mark = np.ascontiguousarray(mark, np.uint8)
    s = _cbg(b)
    lib().orc_bg_size(ctypes.byref(P), ctypes.byref(B), ctypes.byref(s),
                      mark.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))


def bg_split(P, b, next_id):
    s = _cbg(b)
    nid = ctypes.c_longlong(int(next_id))
    r = lib().orc_bg_split(ctypes.byref(P), ctypes.byref(s), ctypes.byref(nid))
    _sync_bg(b, s)
    return r, nid.value


def bg_hsmooth(P, B, b):
    s = _cbg(b)
    lib().orc_bg_hsmooth(ctypes.byref(P), ctypes.byref(B), ctypes.byref(s))


def bg_shift(P, b):
    s = _cbg(b)
    lib().orc_bg_shift(ctypes.byref(P), ctypes.byref(s))


def bg_iteration(P, B, b, next_id, solid, fluid=None):
    """One construction iteration in place; returns (status, stats,
    next_id)."""
    (nw, wx, wy, wh), (nf, fx, fy, fh, phi) = _solid_fluid(solid, fluid)
    s = _cbg(b)
    nid = ctypes.c_longlong(int(next_id))
    z = _BgStats()
    r = lib().orc_bg_iteration(ctypes.byref(P), ctypes.byref(B), ctypes.byref(s),
                               ctypes.byref(nid), nw, _d(wx), _d(wy), _d(wh),
                               nf, _d(fx), _d(fy), _d(fh),
                               _d(phi) if phi is not None else None,
                               ctypes.byref(z))
    _sync_bg(b, s)
    return r, {k: getattr(z, k) for k, _ in _BgStats._fields_}, nid.value


def bg_build(P, B, b, solid, iterations=None, next_id=None, fluid=None):
    """The whole construction: ``iterations`` (default 3 ceil(log(ds_max /
    ds_min) / log Cr)) iterations in place; returns (status, list of
    per-iteration stats, next_id)."""
    if iterations is None:
        iterations = bg_iterations(B)
    if next_id is None:
        next_id = int(b["id"][:b["n"]].max()) + 1 if b["n"] else 0
    stats = []
    for _ in range(iterations):
        r, z, next_id = bg_iteration(P, B, b, next_id, solid, fluid)
        stats.append(z)
        if r != 0:
            return r, stats, next_id
    return 0, stats, next_id
