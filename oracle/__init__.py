"""Plain C oracle of the digital-twin-brain step, with a ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2308_01241_gb300``) never does.

The C source (``dtb_oracle.c``) is compiled twice, with ``REAL=float`` and with
``REAL=double``.  What it computes, with the paper passages it follows:

* Eq. 1 (section III.B): LIF membrane with four conductance receptors
  (AMPA, NMDA, GABAa, GABAb), jump-and-decay gating variables, threshold,
  reset and refractory period;
* section VI.A: explicit (forward) Euler steps;
* section V.D: fixed in-degree connection tables (pull form), turned here
  into outgoing lists for delivery;
* section V.E (citing Friston 2000): Balloon-Windkessel hemodynamics -> BOLD;
* section III.B: external Poisson drive, here by Philox4x32-10 (Salmon et al.
  2011) and exact integer inversion thresholds;
* section III.B: optional Ornstein-Uhlenbeck background current per neuron
  (Euler-Maruyama, Irwin-Hall normals from the same Philox stream family).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "dtb_oracle.c")

NP = 19
P_C, P_GL, P_EL, P_VTH, P_VRESET, P_TREF, P_G, P_TAU, P_E, P_IEXT = 0, 1, 2, 3, 4, 5, 6, 10, 14, 18
W_INT16, W_INT32, W_BF16, W_INT8 = 0, 1, 2, 3
TAG_DRIVE, TAG_INIT, TAG_OU = 1, 2, 3

_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


def lib_path(prec: str) -> str:
    return os.path.join(BUILD_DIR, f"liboracle_{prec}.so")


def build(force: bool = False) -> None:
    """Compile both builds with gcc: no FMA contraction, no fast math."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    hdr = os.path.join(HERE, "dtb_oracle.h")
    for prec, real in (("f32", "float"), ("f64", "double")):
        out = lib_path(prec)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(SRC), os.path.getmtime(hdr)
        ):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-fno-strict-aliasing", f"-DREAL={real}", f"-DORC_SUFFIX=_{prec}",
            "-I", HERE, SRC, "-o", tmp, "-lm",
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


class Desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("n_vox", ctypes.c_int32),
        ("n_ch", ctypes.c_int32),
        ("voxel_start", ctypes.c_void_p),
        ("vparams", ctypes.c_void_p),
        ("dt", ctypes.c_double),
        ("nu_ext", ctypes.c_double),
        ("w_ext", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("pre", ctypes.c_void_p),
        ("cls", ctypes.c_void_p),
        ("wfmt", ctypes.c_int32),
        ("w", ctypes.c_void_p),
        ("wshift", ctypes.c_int32),
        ("pre_shift", ctypes.c_void_p),
        ("delay_vv", ctypes.c_void_p),
        ("d_max", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("init_seed", ctypes.c_uint64),
        ("bold_eps", ctypes.c_double),
        ("bold_tau_s", ctypes.c_double),
        ("bold_tau_f", ctypes.c_double),
        ("bold_tau_0", ctypes.c_double),
        ("bold_alpha", ctypes.c_double),
        ("bold_E0", ctypes.c_double),
        ("bold_V0", ctypes.c_double),
        ("index_base", ctypes.c_int64),
        ("ou_enable", ctypes.c_int32),
        ("ou_mu", ctypes.c_double),
        ("ou_sigma", ctypes.c_double),
        ("ou_tau", ctypes.c_double),
    ]


class BoldParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("eps", "tau_s", "tau_f", "tau_0", "alpha", "E0", "V0")]


def _load(prec: str) -> ctypes.CDLL:
    with _lock:
        if prec in _libs:
            return _libs[prec]
        build()
        lib = ctypes.CDLL(lib_path(prec))
        s = "_" + prec
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
        lib.orc_philox4x32_10.restype = None
        lib.orc_poisson_thresholds.argtypes = [ctypes.c_double, vp, ctypes.c_int]
        lib.orc_poisson_thresholds.restype = ctypes.c_int
        lib.orc_error.restype = ctypes.c_char_p
        lib.orc_drive_counts.argtypes = [ctypes.c_uint64, ctypes.c_double, i64, i64, i64, vp]
        lib.orc_drive_counts.restype = ctypes.c_int
        lib.orc_bold_integrate.argtypes = [ctypes.POINTER(BoldParams), i32, vp, i64, ctypes.c_double, vp, vp]
        lib.orc_bold_integrate.restype = None
        lib.orc_enkf.argtypes = [vp, vp, vp, vp, vp, i32, i32, ctypes.c_double]
        lib.orc_enkf.restype = ctypes.c_int
        lib.orc_deliver_pull.argtypes = [ctypes.POINTER(Desc), i64, vp, vp, vp, vp, vp, i64, vp]
        lib.orc_deliver_pull.restype = ctypes.c_int
        getattr(lib, "orc_create" + s).argtypes = [ctypes.POINTER(Desc)]
        getattr(lib, "orc_create" + s).restype = vp
        getattr(lib, "orc_destroy" + s).argtypes = [vp]
        getattr(lib, "orc_run" + s).argtypes = [vp, i64, vp, i64, vp]
        getattr(lib, "orc_run" + s).restype = i64
        getattr(lib, "orc_get_state" + s).argtypes = [vp, vp, vp, vp, vp, vp]
        getattr(lib, "orc_set_state" + s).argtypes = [vp, vp, vp, vp, vp, i64]
        getattr(lib, "orc_get_bold" + s).argtypes = [vp, vp, vp]
        getattr(lib, "orc_set_g" + s).argtypes = [vp, vp]
        getattr(lib, "orc_get_ou" + s).argtypes = [vp, vp]
        getattr(lib, "orc_events" + s).argtypes = [vp]
        getattr(lib, "orc_events" + s).restype = i64
        _libs[prec] = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter and 2-word key (Salmon et al. 2011)."""
    lib = _load("f32")
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def poisson_thresholds(lam: float) -> np.ndarray:
    """Inversion thresholds floor(2^32 * P(K <= m)) of Poisson(lam)."""
    lib = _load("f32")
    T = np.zeros(64, dtype=np.uint32)
    M = lib.orc_poisson_thresholds(float(lam), _ptr(T), 64)
    if M < 0:
        raise ValueError("bad Poisson rate")
    return T[:M].copy()


def drive_counts(seed: int, lam: float, t: int, i0: int, cnt: int) -> np.ndarray:
    """Poisson drive counts of neurons [i0, i0+cnt) at step t."""
    lib = _load("f32")
    k = np.zeros(cnt, np.int32)
    if lib.orc_drive_counts(int(seed), float(lam), int(t), int(i0), int(cnt), _ptr(k)) != 0:
        raise ValueError("bad drive rate")
    return k


def bold_integrate(params: dict, z, n_steps: int, dt_s: float, state=None):
    """Balloon-Windkessel Euler integration at constant rates z; returns (state [4][nv], y [nv])."""
    lib = _load("f64")
    z = np.ascontiguousarray(z, np.float64)
    nv = z.size
    if state is None:
        state = np.zeros((4, nv), np.float64)
        state[1:] = 1.0
    state = np.ascontiguousarray(state, np.float64).copy()
    y = np.zeros(nv, np.float64)
    p = BoldParams(**{k: float(params[k]) for k in ("eps", "tau_s", "tau_f", "tau_0", "alpha", "E0", "V0")})
    lib.orc_bold_integrate(ctypes.byref(p), nv, _ptr(z), int(n_steps), float(dt_s), _ptr(state), _ptr(y))
    return state, y


def enkf(theta, hx, y, sd, eps, lam: float = 1.0) -> np.ndarray:
    """Stochastic EnKF analysis, local per column: theta, hx, eps [C][M]; y, sd [C].
    Returns the updated theta (double)."""
    lib = _load("f64")
    th = np.ascontiguousarray(theta, np.float64).copy()
    C, M = th.shape
    hx = np.ascontiguousarray(hx, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    sd = np.ascontiguousarray(np.broadcast_to(sd, (C,)), np.float64)
    eps = np.ascontiguousarray(eps, np.float64)
    if lib.orc_enkf(_ptr(th), _ptr(hx), _ptr(y), _ptr(sd), _ptr(eps), C, M, float(lam)) != 0:
        raise ValueError("need at least two members")
    return th


def deliver_pull(net: dict, tgt, pre, cls, w, fired, t: int) -> np.ndarray:
    """Pull-form delivery for targets tgt [m] with rows pre/cls/w [m][K] of a
    network dict (voxel_start, delay_vv, d_max, n_ch, wfmt, wshift, n, K):
    returns int64 acc [m][n_ch][D] of the spikes fired [n] (uint8) at step t."""
    lib = _load("f32")
    tgt = np.ascontiguousarray(tgt, np.int64)
    m = tgt.size
    K = int(net["K"])
    wdt = {W_INT16: np.int16, W_INT32: np.int32, W_BF16: np.uint16, W_INT8: np.int8}[int(net["wfmt"])]
    pre = np.ascontiguousarray(pre, np.int32).reshape(m, K)
    cls = np.ascontiguousarray(cls, np.uint8).reshape(m, K)
    w = np.ascontiguousarray(w, wdt).reshape(m, K)
    fired = np.ascontiguousarray(fired, np.uint8)
    vs = np.ascontiguousarray(net["voxel_start"], np.int64)
    dl = np.ascontiguousarray(net["delay_vv"], np.uint8)
    ps = None if net.get("pre_shift") is None else np.ascontiguousarray(net["pre_shift"], np.uint8)
    d = Desc()
    d.n, d.n_vox, d.n_ch, d.K = int(net["n"]), len(vs) - 1, int(net["n_ch"]), K
    d.voxel_start, d.delay_vv, d.d_max = vs.ctypes.data, dl.ctypes.data, int(net["d_max"])
    d.wfmt, d.wshift = int(net["wfmt"]), int(net["wshift"])
    d.pre_shift = None if ps is None else ps.ctypes.data
    D = d.d_max + 1
    acc = np.zeros((m, d.n_ch, D), np.int64)
    r = lib.orc_deliver_pull(ctypes.byref(d), m, _ptr(tgt), _ptr(pre), _ptr(cls), _ptr(w), _ptr(fired), int(t),
                             _ptr(acc))
    if r != 0:
        raise ValueError("bad pull rows")
    return acc


class OracleNet:
    """One oracle network.  ``prec`` is "f32" (bit-exact reference) or "f64".

    ``net`` is a dict of numpy arrays in the pull form (section V.D):
    ``voxel_start`` int64[V+1], ``vparams`` float64[V][19], ``pre`` int32[n][K],
    ``cls`` uint8[n][K], ``w`` (int16 / int32 / uint16-bf16 / int8)[n][K],
    ``delay_vv`` uint8[V][V] and scalars (see ``Desc``)."""

    def __init__(self, net: dict, prec: str = "f32"):
        self.prec = prec
        self.lib = _load(prec)
        self.real = np.float32 if prec == "f32" else np.float64
        self._s = "_" + prec
        keep = {}

        def arr(name, dtype):
            a = np.ascontiguousarray(net[name], dtype=dtype)
            keep[name] = a
            return a.ctypes.data

        n = int(net["n"])
        K = int(net["K"])
        wdt = {W_INT16: np.int16, W_INT32: np.int32, W_BF16: np.uint16, W_INT8: np.int8}[int(net["wfmt"])]
        d = Desc()
        d.n, d.n_vox, d.n_ch = n, int(net["n_vox"]), int(net["n_ch"])
        d.voxel_start = arr("voxel_start", np.int64)
        d.vparams = arr("vparams", np.float64)
        d.dt, d.nu_ext, d.w_ext, d.K = float(net["dt"]), float(net["nu_ext"]), int(net["w_ext"]), K
        if n * K > 0:
            d.pre = arr("pre", np.int32)
            d.cls = arr("cls", np.uint8)
            d.w = arr("w", wdt)
        d.wfmt, d.wshift = int(net["wfmt"]), int(net["wshift"])
        if net.get("pre_shift") is not None:
            d.pre_shift = arr("pre_shift", np.uint8)
        d.delay_vv = arr("delay_vv", np.uint8)
        d.d_max = int(net["d_max"])
        d.seed, d.init_seed = int(net["seed"]), int(net["init_seed"])
        b = net.get("bold", {})
        d.bold_eps = float(b.get("eps", 0.02))
        d.bold_tau_s = float(b.get("tau_s", 0.8))
        d.bold_tau_f = float(b.get("tau_f", 0.4))
        d.bold_tau_0 = float(b.get("tau_0", 1.0))
        d.bold_alpha = float(b.get("alpha", 0.32))
        d.bold_E0 = float(b.get("E0", 0.34))
        d.bold_V0 = float(b.get("V0", 0.02))
        d.index_base = int(net.get("index_base", 0))
        ou = net.get("ou")
        if ou:
            d.ou_enable, d.ou_mu, d.ou_sigma, d.ou_tau = 1, float(ou["mu"]), float(ou["sigma"]), float(ou["tau"])
        self.n, self.n_vox, self.n_ch, self.D = n, d.n_vox, d.n_ch, d.d_max + 1
        h = getattr(self.lib, "orc_create" + self._s)(ctypes.byref(d))
        if not h:
            raise ValueError("oracle create failed: " + self.lib.orc_error().decode())
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            getattr(self.lib, "orc_destroy" + self._s)(h)
            self.h = None

    def run(self, n_steps: int, ids_cap: int | None = None):
        """Runs n_steps; returns (ids int32[], step_off int64[n_steps+1])."""
        cap = ids_cap if ids_cap is not None else max(1024, self.n * n_steps // 20 + 1024)
        while True:
            ids = np.zeros(cap, dtype=np.int32)
            off = np.zeros(n_steps + 1, dtype=np.int64)
            snap = self.get_state()
            r = getattr(self.lib, "orc_run" + self._s)(self.h, n_steps, _ptr(ids), cap, _ptr(off))
            if r >= 0:
                return ids[:r].copy(), off
            msg = self.lib.orc_error().decode()
            if "spike buffer" not in msg:
                raise RuntimeError("oracle run failed: " + msg)
            self.set_state(*snap)
            cap *= 4

    def get_state(self):
        n = self.n
        V = np.zeros(n, self.real)
        j = np.zeros((4, n), self.real)
        ref = np.zeros(n, np.uint8)
        ring = np.zeros((self.D, self.n_ch, n), np.int32)
        t = np.zeros(1, np.int64)
        getattr(self.lib, "orc_get_state" + self._s)(self.h, _ptr(V), _ptr(j), _ptr(ref), _ptr(ring), _ptr(t))
        return V, j, ref, ring, int(t[0])

    def set_state(self, V, j, ref, ring, t):
        V = np.ascontiguousarray(V, self.real)
        j = np.ascontiguousarray(j, self.real)
        ref = np.ascontiguousarray(ref, np.uint8)
        ring = np.ascontiguousarray(ring, np.int32)
        getattr(self.lib, "orc_set_state" + self._s)(self.h, _ptr(V), _ptr(j), _ptr(ref), _ptr(ring), int(t))

    def get_bold(self):
        y = np.zeros(self.n_vox, np.float64)
        st = np.zeros((4, self.n_vox), np.float64)
        getattr(self.lib, "orc_get_bold" + self._s)(self.h, _ptr(y), _ptr(st))
        return y, st

    def get_ou(self):
        I = np.zeros(self.n, self.real)
        getattr(self.lib, "orc_get_ou" + self._s)(self.h, _ptr(I))
        return I

    def set_g(self, g):
        g = np.ascontiguousarray(g, np.float64).reshape(self.n_vox, 4)
        getattr(self.lib, "orc_set_g" + self._s)(self.h, _ptr(g))

    def events(self) -> int:
        return int(getattr(self.lib, "orc_events" + self._s)(self.h))
