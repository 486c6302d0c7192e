"""ctypes binding of libdtb.so (``include/dtb.h``): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels.  PyTorch is
used for device memory (the library's allocator hooks call into torch's
caching allocator) and for the CUDA stream the work is queued on.  If the
library is missing this module raises at import time: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")

_lib = ctypes.CDLL(LIB_PATH)

DTB_OK, DTB_EINVAL, DTB_ENOMEM, DTB_ECUDA, DTB_EOVERFLOW, DTB_ETIMEOUT, DTB_ETRUNC, DTB_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
W_INT16, W_INT32, W_BF16, W_INT8 = 0, 1, 2, 3
WFMT = {"int16": W_INT16, "int32": W_INT32, "bf16": W_BF16, "int8": W_INT8}
DELIVER_RING, DELIVER_QUEUE, DELIVER_BINS = 0, 1, 2
DELIVERY = {"ring": DELIVER_RING, "queue": DELIVER_QUEUE, "bins": DELIVER_BINS}
# dtb_profile_steps' five entries; the fourth is the queue drain (queue mode)
# or the binning of the step's arrivals (bins mode)
KERNELS = ("neuron_update", "spike_compact", "spike_deliver", "queue_drain", "bold_step")
NP = 19

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class dtb_network_desc(ctypes.Structure):  # noqa: N801 (C name)
    _fields_ = [
        ("n_neurons", ctypes.c_int64), ("n_voxels", ctypes.c_int32), ("n_channels", ctypes.c_int32),
        ("voxel_start", ctypes.c_void_p), ("voxel_params", ctypes.c_void_p),
        ("dt", ctypes.c_double), ("nu_ext", ctypes.c_double),
        ("w_ext", ctypes.c_int32), ("weight_format", ctypes.c_int32), ("weight_shift", ctypes.c_int32),
        ("d_max", ctypes.c_int32),
        ("row_ptr", ctypes.c_void_p), ("syn_word", ctypes.c_void_p), ("syn_w", ctypes.c_void_p),
        ("row_shift", ctypes.c_void_p), ("csr_on_device", ctypes.c_int32), ("bold_every", ctypes.c_int32),
        ("delay_vv", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("init_seed", ctypes.c_uint64),
        ("bold_eps", ctypes.c_double), ("bold_tau_s", ctypes.c_double), ("bold_tau_f", ctypes.c_double),
        ("bold_tau_0", ctypes.c_double), ("bold_alpha", ctypes.c_double), ("bold_E0", ctypes.c_double),
        ("bold_V0", ctypes.c_double), ("spike_log_capacity", ctypes.c_int64),
        ("delivery_mode", ctypes.c_int32), ("bin_capacity", ctypes.c_int32), ("event_queue_capacity", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
        ("ou_enable", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("ou_mu", ctypes.c_double), ("ou_sigma", ctypes.c_double), ("ou_tau", ctypes.c_double),
    ]


_vp, _i64, _i32, _st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32
_SIGS = {
    "dtb_last_error": ([], ctypes.c_char_p),
    "dtb_create_network": ([ctypes.POINTER(dtb_network_desc), ctypes.POINTER(ctypes.c_void_p)], _st),
    "dtb_destroy": ([_vp], _st),
    "dtb_step": ([_vp, _i64], _st),
    "dtb_get_spikes": ([_vp, _vp, _vp, _i64, _vp], _st),
    "dtb_get_bold": ([_vp, _vp, _vp], _st),
    "dtb_get_bold_samples": ([_vp, _vp, _i64, _vp], _st),
    "dtb_get_state": ([_vp, _vp, _vp, _vp, _vp, _vp], _st),
    "dtb_set_state": ([_vp, _vp, _vp, _vp, _vp, _i64], _st),
    "dtb_reset": ([_vp], _st),
    "dtb_set_hyperparams": ([_vp, _vp], _st),
    "dtb_counters": ([_vp, _vp, _vp, _vp], _st),
    "dtb_profile_steps": ([_vp, _i64, _vp], _st),
    "dtb_step_timed": ([_vp, _i64, _vp, _vp], _st),
    "dtb_get_ou": ([_vp, _vp], _st),
    "dtb_set_ou": ([_vp, _vp], _st),
    "dtb_save_state": ([_vp, _vp, ctypes.c_size_t, _vp], _st),
    "dtb_load_state": ([_vp, _vp, ctypes.c_size_t], _st),
    "dtb_philox_device": ([_vp, _vp, _vp, _i64, _vp], _st),
    "dtb_ring_slot_sums": ([_vp, _vp], _st),
    "dtb_get_voxel_spikes": ([_vp, _vp], _st),
    "dtb_autotune": ([_vp, _i32, _vp], _st),
    "dtb_set_launch_shapes": ([_vp, _i32, _i32, _i32], _st),
    "dtb_set_schedule": ([_vp, _i32], _st),
    "dtb_get_schedule": ([_vp, _vp], _st),
    "dtb_bounded_wait_test": ([_i64, _i32], _st),
    "dtb_test_preset_counters": ([_vp, ctypes.c_uint64], _st),
    "dtb_enkf_analysis": ([_vp, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_float, _vp], _st),
    "dtb_ensemble_create": ([_vp, _vp, ctypes.POINTER(ctypes.c_void_p)], _st),
    "dtb_ensemble_destroy": ([_vp], _st),
    "dtb_ensemble_get_theta": ([_vp, _vp], _st),
    "dtb_assimilate": ([_vp, _vp, _i32, _vp, _vp, _vp], _st),
    "dtb_spike_compact": ([_vp, _i64, _vp, _vp, _vp], _st),
    "dtb_spike_compact_noalloc": ([_vp, _i64, _vp, _vp, _vp], _st),
    "dtb_get_ring_at": ([_vp, _vp, _i64, _vp], _st),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class DtbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed ({code}): {_lib.dtb_last_error().decode()}")


def _check(code: int, where: str) -> int:
    if code != DTB_OK:
        raise DtbError(code, where)
    return code


def _p(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# thin wrappers with the C names ------------------------------------------------
def dtb_last_error() -> str:
    return _lib.dtb_last_error().decode()


def dtb_create_network(desc: dtb_network_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.dtb_create_network(ctypes.byref(desc), ctypes.byref(h)), "dtb_create_network")
    return h.value


def dtb_destroy(h) -> None:
    _check(_lib.dtb_destroy(h), "dtb_destroy")


def dtb_step(h, n_steps: int) -> None:
    _check(_lib.dtb_step(h, int(n_steps)), "dtb_step")


def dtb_philox_device(ctr, key, out, stream=None) -> None:
    """Device Philox of torch int32 tensors ctr [n][4], key [n][2] -> out [n][4]."""
    _check(_lib.dtb_philox_device(ctr.data_ptr(), key.data_ptr(), out.data_ptr(), ctr.shape[0], stream),
           "dtb_philox_device")


def dtb_spike_compact(bits, n: int, ids, count, stream=None) -> None:
    """Ascending ids of the set bits of device tensor bits (int32 [ceil(n/1024)*32])
    into ids (int32 [n]); the count into the one-element device tensor count."""
    _check(_lib.dtb_spike_compact(bits.data_ptr(), int(n), ids.data_ptr(), count.data_ptr(), stream),
           "dtb_spike_compact")


def dtb_enkf_analysis(theta, hx, y, obs_sd, eps, inflation: float = 1.0, stream=None) -> None:
    """EnKF analysis on float32 device tensors theta, hx, eps [C][M], y, obs_sd [C] (theta in place)."""
    C, M = theta.shape
    _check(_lib.dtb_enkf_analysis(theta.data_ptr(), hx.data_ptr(), y.data_ptr(), obs_sd.data_ptr(), eps.data_ptr(),
                                  int(C), int(M), float(inflation), stream), "dtb_enkf_analysis")


class dtb_ensemble_desc(ctypes.Structure):  # noqa: N801 (C name)
    _fields_ = [
        ("n_columns", ctypes.c_int32), ("n_members", ctypes.c_int32),
        ("member_voxel", ctypes.c_void_p), ("target_voxel", ctypes.c_void_p), ("theta0", ctypes.c_void_p),
        ("g_base", ctypes.c_void_p), ("receptor_mask", ctypes.c_int32), ("tr_steps", ctypes.c_int32),
        ("obs_sd_rel", ctypes.c_float), ("inflation", ctypes.c_float), ("seed", ctypes.c_uint64),
    ]


class Assimilation:
    """An assimilation ensemble over a Network (dtb_ensemble): member and
    target voxels per column, run by dtb_assimilate."""

    def __init__(self, net, member_voxel, theta0, g_base, tr_steps, target_voxel=None, receptor_mask=0,
                 obs_sd_rel=0.02, inflation=1.0, seed=0):
        self.net = net
        mv = np.ascontiguousarray(member_voxel, np.int32)
        self.C, self.M = mv.shape
        th = np.ascontiguousarray(theta0, np.float32).reshape(self.C, self.M)
        gb = np.ascontiguousarray(g_base, np.float64).reshape(net.n_vox, 4)
        tv = None if target_voxel is None else np.ascontiguousarray(target_voxel, np.int32).reshape(self.C)
        d = dtb_ensemble_desc()
        d.n_columns, d.n_members = self.C, self.M
        d.member_voxel, d.theta0, d.g_base = mv.ctypes.data, th.ctypes.data, gb.ctypes.data
        d.target_voxel = None if tv is None else tv.ctypes.data
        d.receptor_mask, d.tr_steps = int(receptor_mask), int(tr_steps)
        d.obs_sd_rel, d.inflation, d.seed = float(obs_sd_rel), float(inflation), int(seed)
        h = ctypes.c_void_p()
        _check(_lib.dtb_ensemble_create(net.h, ctypes.byref(d), ctypes.byref(h)), "dtb_ensemble_create")
        self.h = h.value
        self.tr_steps = int(tr_steps)

    def close(self):
        if getattr(self, "h", None):
            _check(_lib.dtb_ensemble_destroy(self.h), "dtb_ensemble_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def theta(self) -> np.ndarray:
        th = np.zeros((self.C, self.M), np.float32)
        _check(_lib.dtb_ensemble_get_theta(self.h, th.ctypes.data), "dtb_ensemble_get_theta")
        return th

    def assimilate(self, n_tr: int, bold_obs=None, history: bool = True):
        """n_tr cycles; returns (theta_hist [n_tr][C][M], hx_hist, y_hist [n_tr][C]) or Nones."""
        obs = None if bold_obs is None else np.ascontiguousarray(bold_obs, np.float32).reshape(n_tr, self.C)
        th = np.zeros((n_tr, self.C, self.M), np.float32) if history else None
        hx = np.zeros((n_tr, self.C, self.M), np.float32) if history else None
        y = np.zeros((n_tr, self.C), np.float32) if history else None
        _check(_lib.dtb_assimilate(self.h, _p(obs), int(n_tr), _p(th), _p(hx), _p(y)), "dtb_assimilate")
        self.net._nsteps = self.tr_steps
        return th, hx, y


NOALLOC_MAX_NEURONS = 1 << 28


def dtb_spike_compact_noalloc(bits, n: int, ids, count, stream=None) -> None:
    """dtb_spike_compact without any device allocation (fixed library scratch,
    n <= NOALLOC_MAX_NEURONS; concurrent calls on the GPU race)."""
    _check(_lib.dtb_spike_compact_noalloc(bits.data_ptr(), int(n), ids.data_ptr(), count.data_ptr(), stream),
           "dtb_spike_compact_noalloc")


class _TorchAllocator:
    """Device memory for the library from torch's caching allocator."""

    def __init__(self, device):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, p, ctx):
        self.live.pop(p, None)


class Network:
    """One simulated network on one GPU (a dtb_net handle).

    csr: (row_ptr, syn_word, syn_w[, row_shift]) either host numpy arrays or
    device torch tensors (used in place, kept alive by this object)."""

    def __init__(self, *, n, voxel_start, vparams, delay_vv, d_max, csr, wfmt="int16", wshift=4, n_ch=2,
                 dt=0.1, nu_ext=2000.0, w_ext=65536, seed=2, init_seed=3, bold=None, bold_every=8000,
                 log_capacity=0, delivery="ring", event_queue_capacity=0, bin_capacity=0, ou=None,
                 device="cuda:0"):
        """ou: None, or dict(mu=nA, sigma=nA, tau=ms) for the Ornstein-Uhlenbeck background current."""
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(device=self.device)
        self._alloc = _TorchAllocator(self.device)
        self._keep = []
        bold = bold or {}
        self.n, self.n_vox, self.n_ch, self.D = int(n), len(voxel_start) - 1, int(n_ch), int(d_max) + 1
        self._nsteps = 0
        keep = self._keep

        def host(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        d = dtb_network_desc()
        d.n_neurons, d.n_voxels, d.n_channels = self.n, self.n_vox, self.n_ch
        d.voxel_start = host(voxel_start, np.int64)
        d.voxel_params = host(np.asarray(vparams, np.float64).reshape(self.n_vox, NP), np.float64)
        d.dt, d.nu_ext, d.w_ext = float(dt), float(nu_ext), int(w_ext)
        d.weight_format = WFMT[wfmt] if isinstance(wfmt, str) else int(wfmt)
        d.weight_shift, d.d_max = int(wshift), int(d_max)
        on_dev = not isinstance(csr[0], np.ndarray)
        if on_dev:
            keep.extend(csr)
            d.row_ptr, d.syn_word, d.syn_w = (c.data_ptr() for c in csr[:3])
            d.row_shift = csr[3].data_ptr() if len(csr) > 3 and csr[3] is not None else None
        else:
            d.row_ptr = host(csr[0], np.int64)
            d.syn_word = host(csr[1], np.uint32)
            w = np.ascontiguousarray(csr[2])
            keep.append(w)
            d.syn_w = w.ctypes.data
            d.row_shift = host(csr[3], np.uint8) if len(csr) > 3 and csr[3] is not None else None
        d.csr_on_device = 1 if on_dev else 0
        d.bold_every = int(bold_every)
        d.delay_vv = host(delay_vv, np.uint8)
        d.seed, d.init_seed = int(seed), int(init_seed)
        d.bold_eps = float(bold.get("eps", 0.02))
        d.bold_tau_s = float(bold.get("tau_s", 0.8))
        d.bold_tau_f = float(bold.get("tau_f", 0.4))
        d.bold_tau_0 = float(bold.get("tau_0", 1.0))
        d.bold_alpha = float(bold.get("alpha", 0.32))
        d.bold_E0 = float(bold.get("E0", 0.34))
        d.bold_V0 = float(bold.get("V0", 0.02))
        d.spike_log_capacity = int(log_capacity)
        d.delivery_mode = DELIVERY[delivery] if isinstance(delivery, str) else int(delivery)
        d.event_queue_capacity = int(event_queue_capacity)
        d.bin_capacity = int(bin_capacity)
        d.stream = self.stream.cuda_stream
        d.alloc, d.free, d.alloc_ctx = self._alloc.alloc_cb, self._alloc.free_cb, None
        if ou:
            d.ou_enable, d.ou_mu, d.ou_sigma, d.ou_tau = 1, float(ou["mu"]), float(ou["sigma"]), float(ou["tau"])
        with torch.cuda.device(self.device):
            self.h = dtb_create_network(d)
        self._keep = [k for k in keep if not isinstance(k, np.ndarray)]  # host arrays were copied

    # -- lifecycle
    def close(self) -> None:
        if getattr(self, "h", None):
            dtb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping
    def step(self, n_steps: int) -> None:
        dtb_step(self.h, n_steps)
        self._nsteps = int(n_steps)

    def step_timed(self, n_steps: int):
        """Runs n_steps like step() (same schedule, no graph) with events around
        every kernel: (ms float64[5], launches int64[5]) summed over the body
        steps, in the order of KERNELS."""
        ms = np.zeros(5, np.float64)
        cnt = np.zeros(5, np.int64)
        _check(_lib.dtb_step_timed(self.h, int(n_steps), ms.ctypes.data, cnt.ctypes.data), "dtb_step_timed")
        self._nsteps = int(n_steps)
        return ms, cnt

    def profile_steps(self, n_steps: int) -> np.ndarray:
        """Per-kernel device ms over n_steps, in the order of KERNELS."""
        ms = np.zeros(5, np.float64)
        _check(_lib.dtb_profile_steps(self.h, int(n_steps), ms.ctypes.data), "dtb_profile_steps")
        self._nsteps = int(n_steps)
        return ms

    # -- outputs
    def get_spikes(self, n_steps: int | None = None, ids_out=None, off_out=None):
        """(ids int32[], step_off int64[n_steps+1]) of the last step call.

        n_steps, when given, must be that call's step count; ids_out and
        off_out are optional preallocated host buffers (contiguous int32 with
        room for every id, contiguous int64 with n_steps + 1 entries)."""
        steps = self._nsteps
        if n_steps is not None and int(n_steps) != steps:
            raise ValueError(f"get_spikes: the last step call ran {steps} steps, not {n_steps}")
        n_out = ctypes.c_int64()
        _check_trunc = _lib.dtb_get_spikes(self.h, None, None, 0, ctypes.byref(n_out))
        if _check_trunc not in (DTB_OK, DTB_ETRUNC):
            _check(_check_trunc, "dtb_get_spikes")
        total = n_out.value
        ids = ids_out if ids_out is not None and ids_out.size >= total else np.zeros(max(total, 1), np.int32)
        off = off_out if off_out is not None else np.zeros(steps + 1, np.int64)
        if off.dtype != np.int64 or not off.flags.c_contiguous or off.size < steps + 1:
            raise ValueError(f"get_spikes: off_out needs {steps + 1} contiguous int64 entries")
        if ids.dtype != np.int32 or not ids.flags.c_contiguous:
            raise ValueError("get_spikes: ids_out must be contiguous int32")
        _check(_lib.dtb_get_spikes(self.h, off.ctypes.data, ids.ctypes.data, ids.size, ctypes.byref(n_out)),
               "dtb_get_spikes")
        return ids[:total], off[: steps + 1]

    def get_bold(self):
        y = np.zeros(self.n_vox, np.float32)
        st = np.zeros((4, self.n_vox), np.float32)
        _check(_lib.dtb_get_bold(self.h, y.ctypes.data, st.ctypes.data), "dtb_get_bold")
        return y, st

    def get_bold_samples(self):
        k = ctypes.c_int64()
        _check(_lib.dtb_get_bold_samples(self.h, None, 0, ctypes.byref(k)), "dtb_get_bold_samples")
        out = np.zeros((max(k.value, 1), self.n_vox), np.float32)
        _check(_lib.dtb_get_bold_samples(self.h, out.ctypes.data, out.shape[0], ctypes.byref(k)),
               "dtb_get_bold_samples")
        return out[: k.value]

    def get_state(self, with_ring: bool = True):
        """(V [n], j [4][n], ref [n], ring [D][n_ch][n] or None, t)."""
        n = self.n
        V = np.zeros(n, np.float32)
        j = np.zeros((4, n), np.float32)
        ref = np.zeros(n, np.uint8)
        ring = np.zeros((self.D, self.n_ch, n), np.int32) if with_ring else None
        t = ctypes.c_int64()
        _check(_lib.dtb_get_state(self.h, V.ctypes.data, j.ctypes.data, ref.ctypes.data, _p(ring),
                                  ctypes.byref(t)), "dtb_get_state")
        return V, j, ref, ring, t.value

    def ring_slot_sums(self) -> np.ndarray:
        """int64 [D][n_ch] sums of the delay ring, computed on the device."""
        s = np.zeros((self.D, self.n_ch), np.int64)
        _check(_lib.dtb_ring_slot_sums(self.h, s.ctypes.data), "dtb_ring_slot_sums")
        return s

    def get_ring_at(self, idx) -> np.ndarray:
        """int32 [m][D][n_ch] ring entries of neurons idx."""
        idx = np.ascontiguousarray(idx, np.int64)
        out = np.zeros((idx.size, self.D, self.n_ch), np.int32)
        _check(_lib.dtb_get_ring_at(self.h, idx.ctypes.data, idx.size, out.ctypes.data), "dtb_get_ring_at")
        return out

    def set_state(self, V=None, j=None, ref=None, ring=None, t=0) -> None:
        """V [n], j [4][n], ref [n], ring [D][n_ch][n] (None: left as is), step t."""
        n = self.n
        shapes = ((n,), (4, n), (n,), (self.D, self.n_ch, n))
        a = []
        for x, dt, shape, name in zip((V, j, ref, ring), (np.float32, np.float32, np.uint8, np.int32), shapes,
                                      ("V", "j", "ref", "ring")):
            if x is not None:
                x = np.ascontiguousarray(x, dt)
                if x.shape != shape:
                    raise ValueError(f"set_state: {name} has shape {x.shape}, expected {shape}")
            a.append(x)
        _check(_lib.dtb_set_state(self.h, *[_p(x) for x in a], int(t)), "dtb_set_state")
        self._nsteps = 0

    def reset(self) -> None:
        _check(_lib.dtb_reset(self.h), "dtb_reset")
        self._nsteps = 0

    def set_hyperparams(self, g) -> None:
        g = np.ascontiguousarray(g, np.float64).reshape(self.n_vox, 4)
        _check(_lib.dtb_set_hyperparams(self.h, g.ctypes.data), "dtb_set_hyperparams")

    def autotune(self, n_steps: int = 50) -> dict:
        """Picks launch shapes by timing (advances the state: reset afterwards)."""
        c = np.zeros(3, np.int32)
        _check(_lib.dtb_autotune(self.h, int(n_steps), c.ctypes.data), "dtb_autotune")
        self._nsteps = 0
        return {"update_stages": int(c[0]), "update_ctas_per_sm": int(c[1]), "deliver_ctas_per_sm": int(c[2])}

    def get_ou(self) -> np.ndarray:
        """float32 [n] OU currents (the OU drive must be on)."""
        I = np.zeros(self.n, np.float32)
        _check(_lib.dtb_get_ou(self.h, I.ctypes.data), "dtb_get_ou")
        return I

    def set_ou(self, I) -> None:
        I = np.ascontiguousarray(I, np.float32).reshape(self.n)
        _check(_lib.dtb_set_ou(self.h, I.ctypes.data), "dtb_set_ou")

    def set_shapes(self, update_stages: int, update_ctas_per_sm: int, deliver_ctas_per_sm: int) -> None:
        """Launch shapes (the autotuner's choices) set by hand."""
        _check(_lib.dtb_set_launch_shapes(self.h, int(update_stages), int(update_ctas_per_sm),
                                          int(deliver_ctas_per_sm)), "dtb_set_launch_shapes")

    def set_schedule(self, mode: int) -> None:
        """-1 by size (default), 0 compaction after the update, 1 compaction beside the next update."""
        _check(_lib.dtb_set_schedule(self.h, int(mode)), "dtb_set_schedule")

    def schedule_beside(self) -> bool:
        """True when the compaction of a step runs beside the next step's update."""
        b = ctypes.c_int32(0)
        _check(_lib.dtb_get_schedule(self.h, ctypes.byref(b)), "dtb_get_schedule")
        return bool(b.value)

    def test_preset_counters(self, value: int) -> None:
        """Test hook: every queue and bin count set to value, unused entries weight-0 placeholders."""
        _check(_lib.dtb_test_preset_counters(self.h, int(value)), "dtb_test_preset_counters")

    def voxel_spikes(self) -> np.ndarray:
        """int64 [n_vox] spikes per voxel since creation or reset."""
        c = np.zeros(self.n_vox, np.int64)
        _check(_lib.dtb_get_voxel_spikes(self.h, c.ctypes.data), "dtb_get_voxel_spikes")
        return c

    def counters(self):
        ev, sp, st = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.dtb_counters(self.h, ctypes.byref(ev), ctypes.byref(sp), ctypes.byref(st)), "dtb_counters")
        return ev.value, sp.value, st.value

    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(_lib.dtb_save_state(self.h, None, 0, ctypes.byref(n)), "dtb_save_state")
        buf = ctypes.create_string_buffer(n.value)
        _check(_lib.dtb_save_state(self.h, buf, n.value, ctypes.byref(n)), "dtb_save_state")
        return buf.raw

    def load_state(self, blob: bytes) -> None:
        _check(_lib.dtb_load_state(self.h, blob, len(blob)), "dtb_load_state")
        self._nsteps = 0



def from_tables(tb, csr, rate="default", wfmt=None, device="cuda:0", **kw) -> Network:
    """Network from netgen tables and a CSR (host numpy or device torch)."""
    from .netgen import gain_for

    cfg = tb.cfg
    wfmt = wfmt or cfg["wfmt"]
    kw.setdefault("bold_every", int(cfg["bold"].get("every", 8000)))
    return Network(n=tb.n, voxel_start=tb.voxel_start, vparams=tb.vparams(gain_for(cfg, rate)),
                   delay_vv=tb.delay_vv, d_max=tb.d_max, csr=csr, wfmt=wfmt, wshift=4 if wfmt == "int16" else 0,
                   n_ch=int(cfg["n_ch"]), dt=float(cfg["dt"]), nu_ext=float(cfg["nu_ext"]), w_ext=int(cfg["w_ext"]),
                   seed=int(cfg["seeds"]["drive"]), init_seed=int(cfg["seeds"]["init"]), bold=cfg["bold"],
                   device=device, **kw)


def host_csr(tb, pull, wfmt=None):
    """Host CSR arrays (row_ptr, word, stored weights) from netgen's pull form."""
    from .netgen import host_push

    wfmt = wfmt or tb.cfg["wfmt"]
    row_ptr, word, wbin = host_push(tb, pull)
    return row_ptr, word, tb.wtable(wfmt)[wbin]
