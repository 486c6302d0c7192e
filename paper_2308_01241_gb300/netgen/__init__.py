"""Seeded synthetic voxel-structured networks (the input generator).

This module produces the INPUTS shared by the CPU oracle and the GPU library:
voxel sizes, the DTI-like voxel coupling matrix, voxel-pair delays, per-voxel
neuron parameters and the synapses.  It contains none of the simulated
method's arithmetic.  The per-synapse draws live in ``csrc/netgen_core.h`` and
run identically on the host (``netgen_host.c``, for the oracle's pull form and
for host-staged CSRs) and on the device (``netgen_dev.cu``, for the 20M-neuron
network whose CSR does not fit a host staging copy).

Stand-in for the paper's sMRI/DTI/PET-derived network (section III.B,
Table I), which is not available: heterogeneous log-normal voxel sizes, 80/20
E/I split, fixed in-degree, sparse row-normalised inter-voxel coupling with
log-normal strengths, excitatory-only long-range inputs, delays growing with
the distance between random voxel centres.
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CONFIG_DIR = os.path.join(HERE, "configs")
BUILD_DIR = os.path.join(os.path.dirname(HERE), "_build")
HOST_LIB = os.path.join(BUILD_DIR, "libdtbgen_host.so")
DEV_LIB = os.path.join(BUILD_DIR, "libdtbgen_dev.so")
WBITS = 12
NP = 19  # per-voxel parameter columns (C, gL, EL, Vth, Vreset, t_ref, g[4], tau[4], E[4], I_ext)
WFMT = {"int16": 0, "int32": 1, "bf16": 2, "int8": 3}

_lock = threading.Lock()
_host = None
_dev = None


# ----------------------------------------------------------------------------- build
def build_host(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    src = os.path.join(HERE, "csrc", "netgen_host.c")
    hdr = os.path.join(HERE, "csrc", "netgen_core.h")
    if force or not os.path.exists(HOST_LIB) or os.path.getmtime(HOST_LIB) < max(
        os.path.getmtime(src), os.path.getmtime(hdr)
    ):
        tmp = HOST_LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-I", os.path.join(HERE, "csrc"),
                        src, "-o", tmp], check=True)
        os.replace(tmp, HOST_LIB)
    return HOST_LIB


def dev_build_cmd(arch: str = "sm_103a") -> list[list[str]]:
    """nvcc command that builds the device generator library."""
    src = os.path.join(HERE, "csrc", "netgen_dev.cu")
    num = arch.replace("sm_", "")
    return [["nvcc", "-O3", "-std=c++17", f"-gencode=arch=compute_{num},code={arch}", "-lineinfo",
             "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(HERE, "csrc"), src, "-o", DEV_LIB]]


class DgNet(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("nv", ctypes.c_int32), ("K", ctypes.c_int32), ("K_intra", ctypes.c_int32),
        ("pad_", ctypes.c_int32), ("vstart", ctypes.c_void_p), ("nexc", ctypes.c_void_p),
        ("dti_ptr", ctypes.c_void_p), ("dti_src", ctypes.c_void_p), ("dti_cum", ctypes.c_void_p),
        ("key0", ctypes.c_uint32), ("key1", ctypes.c_uint32),
    ]


def _host_lib():
    global _host
    with _lock:
        if _host is None:
            build_host()
            lib = ctypes.CDLL(HOST_LIB)
            vp = ctypes.c_void_p
            lib.dg_host_pull.argtypes = [ctypes.POINTER(DgNet), ctypes.c_int64, ctypes.c_int64, vp, vp, vp]
            lib.dg_host_transpose.argtypes = [ctypes.c_int64, ctypes.c_int32, vp, vp, vp, vp, vp, vp]
            _host = lib
        return _host


def _dev_lib():
    global _dev
    with _lock:
        if _dev is None:
            if not os.path.exists(DEV_LIB):
                raise RuntimeError("device generator library missing; run __graft_entry__.build()")
            lib = ctypes.CDLL(DEV_LIB)
            vp = ctypes.c_void_p
            lib.dg_dev_build.argtypes = [ctypes.POINTER(DgNet), vp, vp, vp, vp, ctypes.c_int, vp, vp, vp]
            lib.dg_dev_build.restype = ctypes.c_int
            lib.dg_dev_quantize_int8.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
            lib.dg_dev_quantize_int8.restype = ctypes.c_int
            _dev = lib
        return _dev


# ----------------------------------------------------------------------------- config
def load_config(name: str) -> dict:
    """Config by file name (without .json) under configs/, or by path."""
    path = name if os.path.exists(name) else os.path.join(CONFIG_DIR, name + ".json")
    with open(path) as f:
        return json.load(f)


def config_names() -> list[str]:
    return sorted(f[:-5] for f in os.listdir(CONFIG_DIR) if f.endswith(".json"))


@dataclass
class Tables:
    """Voxel-level tables of one network (all host numpy)."""
    cfg: dict
    n: int
    nv: int
    K: int
    K_intra: int
    voxel_start: np.ndarray  # int64[nv+1]
    nexc: np.ndarray         # int64[nv]
    dti_ptr: np.ndarray      # int64[nv+1]
    dti_src: np.ndarray      # int32[]
    dti_cum: np.ndarray      # uint64[]
    delay_vv: np.ndarray     # uint8[nv][nv] (source, target)
    d_max: int
    w_float: np.ndarray      # float64[4096] weight of each quantile bin
    key: tuple = (0, 0)
    _keep: list = field(default_factory=list)

    def dg(self) -> DgNet:
        """ctypes view with HOST pointers."""
        arrs = [np.ascontiguousarray(a) for a in (self.voxel_start, self.nexc, self.dti_ptr, self.dti_src,
                                                  self.dti_cum)]
        self._keep = arrs
        d = DgNet()
        d.n, d.nv, d.K, d.K_intra = self.n, self.nv, self.K, self.K_intra
        d.vstart, d.nexc, d.dti_ptr, d.dti_src, d.dti_cum = (a.ctypes.data for a in arrs)
        d.key0, d.key1 = self.key
        return d

    def vparams(self, gain: float = 1.0) -> np.ndarray:
        """float64[nv][19]; gain multiplies g_AMPA and g_NMDA of every voxel."""
        nr = self.cfg["neuron"]
        row = np.zeros(NP, np.float64)
        row[0], row[1], row[2], row[3], row[4], row[5] = nr["C"], nr["gL"], nr["EL"], nr["Vth"], nr["Vreset"], nr["t_ref"]
        row[6:10] = nr["g"]
        row[10:14] = nr["tau"]
        row[14:18] = nr["E"]
        row[18] = nr["I_ext"]
        P = np.tile(row, (self.nv, 1))
        P[:, 6] *= gain
        P[:, 7] *= gain
        return P

    def wtable(self, fmt: str) -> np.ndarray:
        """Stored weight of each quantile bin in the given storage format."""
        w = self.w_float
        if fmt == "int16":  # 2^-12 fixed point
            return np.clip(np.rint(w * 4096.0), 0, 32767).astype(np.int16)
        if fmt == "int32":  # FP32 weight as 2^-16 fixed point
            return np.rint(w.astype(np.float32).astype(np.float64) * 65536.0).astype(np.int32)
        if fmt == "bf16":
            f = w.astype(np.float32).view(np.uint32).astype(np.uint64)
            rounded = (f + 0x7FFF + ((f >> 16) & 1)) >> 16  # round to nearest even
            return rounded.astype(np.uint16)
        raise ValueError(fmt)

    @property
    def wshift(self) -> int:
        return 4 if self.cfg["wfmt"] == "int16" else 0


def gain_for(cfg: dict, rate) -> float:
    g = cfg.get("gain", {})
    return float(g.get(str(rate), g.get("default", 1.0)))


def _voxel_sizes(cfg: dict, rng: np.random.Generator, n_target: int, nv: int) -> np.ndarray:
    sigma = float(cfg["vox_size_sigma"])
    if nv == 1:
        return np.array([n_target], np.int64)
    raw = np.exp(rng.standard_normal(nv) * sigma - 0.5 * sigma * sigma)
    x = raw / raw.sum() * n_target
    x = np.maximum(x, 16.0)
    x = x / x.sum() * n_target
    sizes = np.floor(x).astype(np.int64)
    rem = n_target - int(sizes.sum())
    order = np.argsort(-(x - sizes), kind="stable")
    sizes[order[:rem]] += 1
    return sizes


def make_tables(cfg: dict, n_neurons: int | None = None, n_vox: int | None = None,
                K: int | None = None) -> Tables:
    """Voxel-level tables from a config (sizes may be overridden for small tests)."""
    n = int(n_neurons if n_neurons is not None else cfg["n_neurons"])
    nv = int(n_vox if n_vox is not None else cfg["n_vox"])
    K = int(K if K is not None else cfg["K"])
    seeds = cfg["seeds"]
    rng = np.random.Generator(np.random.Philox(int(seeds["vox"])))
    sizes = _voxel_sizes(cfg, rng, n, nv)
    if sizes.min() < 2:
        raise ValueError("every voxel needs at least two neurons")
    vstart = np.zeros(nv + 1, np.int64)
    vstart[1:] = np.cumsum(sizes)
    # E neurons are the first floor(frac_exc * n_v) of each voxel (exact integer floor)
    nexc = np.maximum((sizes * int(round(float(cfg["frac_exc"]) * 1000))) // 1000, 1).astype(np.int64)
    K_intra = K if nv == 1 else int(round(K * float(cfg["frac_intra"])))
    # DTI-like coupling: row = target voxel, ~density*(nv-1) random source voxels, log-normal strengths
    ptr = np.zeros(nv + 1, np.int64)
    srcs, cums = [], []
    if nv > 1 and K_intra < K:
        m = max(1, int(round(float(cfg["dti_density"]) * (nv - 1))))
        for v in range(nv):
            others = np.delete(np.arange(nv), v)
            s = np.sort(rng.choice(others, size=m, replace=False))
            strength = np.exp(rng.standard_normal(m) * float(cfg["dti_sigma"]))
            p = strength / strength.sum()
            c = np.floor(np.cumsum(p) * 2.0 ** 32).astype(np.uint64)
            c[-1] = np.uint64(1 << 32)
            srcs.append(s.astype(np.int32))
            cums.append(c)
            ptr[v + 1] = ptr[v] + m
    dti_src = np.concatenate(srcs) if srcs else np.zeros(0, np.int32)
    dti_cum = np.concatenate(cums) if cums else np.zeros(0, np.uint64)
    # delays: 1 inside a voxel, 1 + round((d_max-1) * dist / dist_max) between voxel centres
    d_max = int(cfg["d_max"])
    centres = rng.random((nv, 3))
    dist = np.sqrt(((centres[:, None, :] - centres[None, :, :]) ** 2).sum(-1))
    dmx = dist.max() if nv > 1 else 1.0
    delay = (1 + np.rint((d_max - 1) * dist / dmx)).astype(np.int64)
    np.fill_diagonal(delay, 1)
    delay = np.clip(delay, 1, d_max).astype(np.uint8)
    # weight quantile bins of LogNormal(w_mu, w_sigma)
    from scipy.special import ndtri
    q = (np.arange(1 << WBITS) + 0.5) / float(1 << WBITS)
    w_float = np.exp(float(cfg["w_mu"]) + float(cfg["w_sigma"]) * ndtri(q))
    seed = int(seeds["net"])
    return Tables(cfg=cfg, n=n, nv=nv, K=K, K_intra=K_intra, voxel_start=vstart, nexc=nexc, dti_ptr=ptr,
                  dti_src=dti_src, dti_cum=dti_cum, delay_vv=delay, d_max=d_max, w_float=w_float,
                  key=(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))


@dataclass
class EnsembleLayout:
    """Where each network of a batched ensemble sits in the merged network.
    net_vox[g][k] = (first voxel, voxel count) of copy k of group g; copies
    0..M-1 are the members, copy M is the group's hidden target."""
    groups: int
    members: int
    group_vox: list
    net_vox: list


def make_ensemble_tables(cfg: dict, groups: int | None = None, members: int | None = None,
                         vox_range=None, neuron_range=None) -> tuple[Tables, EnsembleLayout]:
    """One block-diagonal network holding every member and target network of
    a batched ensemble: G groups of uneven size, each M members plus one
    target with the group's voxel sizes, DTI-like coupling and delays; no
    synapse crosses two networks (each network's coupling rows name only its
    own voxels)."""
    G = int(groups if groups is not None else cfg["n_groups"])
    M = int(members if members is not None else cfg["members_per_group"])
    vr = vox_range or cfg["vox_range"]
    nr = neuron_range or cfg["neuron_range"]
    rng = np.random.Generator(np.random.Philox(int(cfg["seeds"]["vox"])))
    K = int(cfg["K"])
    K_intra = int(round(K * float(cfg["frac_intra"])))
    d_max = int(cfg["d_max"])
    sizes_all, ptr, srcs, cums, blocks = [], [0], [], [], []
    group_vox, net_vox = [], []
    v_off = 0
    for g in range(G):
        Vg = int(rng.integers(vr[0], vr[1] + 1))
        Ng = int(rng.integers(nr[0], nr[1] + 1))
        sub = dict(cfg, vox_size_sigma=cfg["vox_size_sigma"])
        sz = _voxel_sizes(sub, rng, Ng, Vg)
        m = max(1, int(round(float(cfg["dti_density"]) * (Vg - 1))))
        rows = []
        for v in range(Vg):
            others = np.delete(np.arange(Vg), v)
            s_ = np.sort(rng.choice(others, size=m, replace=False))
            st = np.exp(rng.standard_normal(m) * float(cfg["dti_sigma"]))
            c = np.floor(np.cumsum(st / st.sum()) * 2.0 ** 32).astype(np.uint64)
            c[-1] = np.uint64(1 << 32)
            rows.append((s_, c))
        centres = rng.random((Vg, 3))
        dist = np.sqrt(((centres[:, None, :] - centres[None, :, :]) ** 2).sum(-1))
        dl = np.clip(1 + np.rint((d_max - 1) * dist / max(dist.max(), 1e-12)), 1, d_max).astype(np.uint8)
        np.fill_diagonal(dl, 1)
        group_vox.append(Vg)
        copies = []
        for k in range(M + 1):
            copies.append((v_off, Vg))
            sizes_all.append(sz)
            for s_, c in rows:
                srcs.append((s_ + v_off).astype(np.int32))
                cums.append(c)
                ptr.append(ptr[-1] + len(s_))
            blocks.append((v_off, dl))
            v_off += Vg
        net_vox.append(copies)
    nv = v_off
    sizes = np.concatenate(sizes_all).astype(np.int64)
    vstart = np.zeros(nv + 1, np.int64)
    vstart[1:] = np.cumsum(sizes)
    nexc = np.maximum((sizes * int(round(float(cfg["frac_exc"]) * 1000))) // 1000, 1).astype(np.int64)
    delay = np.ones((nv, nv), np.uint8)
    for off, dl in blocks:
        delay[off:off + dl.shape[0], off:off + dl.shape[0]] = dl
    from scipy.special import ndtri
    q = (np.arange(1 << WBITS) + 0.5) / float(1 << WBITS)
    w_float = np.exp(float(cfg["w_mu"]) + float(cfg["w_sigma"]) * ndtri(q))
    seed = int(cfg["seeds"]["net"])
    tb = Tables(cfg=cfg, n=int(vstart[-1]), nv=nv, K=K, K_intra=K_intra, voxel_start=vstart, nexc=nexc,
                dti_ptr=np.asarray(ptr, np.int64), dti_src=np.concatenate(srcs), dti_cum=np.concatenate(cums),
                delay_vv=delay, d_max=d_max, w_float=w_float, key=(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    return tb, EnsembleLayout(groups=G, members=M, group_vox=group_vox, net_vox=net_vox)


# ----------------------------------------------------------------------------- host generation
def host_pull(tb: Tables, i0: int = 0, i1: int | None = None):
    """Pull form of neurons [i0, i1): (pre int32, cls uint8, wbin uint16), each [(i1-i0), K]."""
    i1 = tb.n if i1 is None else i1
    m = (i1 - i0) * tb.K
    pre = np.zeros(m, np.int32)
    cls = np.zeros(m, np.uint8)
    wbin = np.zeros(m, np.uint16)
    d = tb.dg()
    r = _host_lib().dg_host_pull(ctypes.byref(d), i0, i1, pre.ctypes.data, cls.ctypes.data, wbin.ctypes.data)
    if r != 0:
        raise ValueError("bad neuron range")
    shape = (i1 - i0, tb.K)
    return pre.reshape(shape), cls.reshape(shape), wbin.reshape(shape)


def host_push(tb: Tables, pull):
    """Outgoing CSR (row_ptr int64[n+1], word uint32[nnz] = target | class << 30, wbin uint16[nnz])."""
    pre, cls, wbin = (np.ascontiguousarray(a) for a in pull)
    nnz = tb.n * tb.K
    row_ptr = np.zeros(tb.n + 1, np.int64)
    word = np.zeros(nnz, np.uint32)
    wb = np.zeros(nnz, np.uint16)
    r = _host_lib().dg_host_transpose(tb.n, tb.K, pre.ctypes.data, cls.ctypes.data, wbin.ctypes.data,
                                      row_ptr.ctypes.data, word.ctypes.data, wb.ctypes.data)
    if r != 0:
        raise ValueError("transpose failed")
    return row_ptr, word, wb


def oracle_inputs(tb: Tables, pull, rate="default", wfmt: str | None = None) -> dict:
    """Dict accepted by oracle.OracleNet (pull form, stored weights)."""
    cfg = tb.cfg
    wfmt = wfmt or cfg["wfmt"]
    pre, cls, wbin = pull
    return dict(
        n=tb.n, n_vox=tb.nv, n_ch=int(cfg["n_ch"]), voxel_start=tb.voxel_start,
        vparams=tb.vparams(gain_for(cfg, rate)), dt=float(cfg["dt"]), nu_ext=float(cfg["nu_ext"]),
        w_ext=int(cfg["w_ext"]), K=tb.K, pre=pre, cls=cls, wfmt=WFMT[wfmt], w=tb.wtable(wfmt)[wbin],
        wshift=4 if wfmt == "int16" else 0, delay_vv=tb.delay_vv, d_max=tb.d_max,
        seed=int(cfg["seeds"]["drive"]), init_seed=int(cfg["seeds"]["init"]), bold=dict(cfg["bold"]),
    )


# ----------------------------------------------------------------------------- device generation
def device_csr(tb: Tables, wfmt: str, device="cuda"):
    """Outgoing CSR built on the device: (row_ptr, word, w) torch tensors."""
    import torch

    lib = _dev_lib()
    dev = torch.device(device)
    nnz = tb.n * tb.K
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    vstart, nexc, dptr = t(tb.voxel_start), t(tb.nexc), t(tb.dti_ptr)
    dsrc = t(tb.dti_src if tb.dti_src.size else np.zeros(1, np.int32))
    dcum = t((tb.dti_cum if tb.dti_cum.size else np.zeros(1, np.uint64)).view(np.int64))
    wt_np = tb.wtable(wfmt)
    wt = t(wt_np.view({1: np.int8, 2: np.int16, 4: np.int32}[wt_np.itemsize]))
    row_ptr = torch.empty(tb.n + 1, dtype=torch.int64, device=dev)
    word = torch.empty(nnz, dtype=torch.int32, device=dev)
    w = torch.empty(nnz, dtype={1: torch.int8, 2: torch.int16, 4: torch.int32}[wt_np.itemsize], device=dev)
    cnt = torch.empty(tb.n, dtype=torch.int32, device=dev)
    fill = torch.empty(tb.n, dtype=torch.int32, device=dev)
    d = DgNet()
    d.n, d.nv, d.K, d.K_intra = tb.n, tb.nv, tb.K, tb.K_intra
    d.vstart, d.nexc, d.dti_ptr = vstart.data_ptr(), nexc.data_ptr(), dptr.data_ptr()
    d.dti_src, d.dti_cum = dsrc.data_ptr(), dcum.data_ptr()
    d.key0, d.key1 = tb.key
    stream = torch.cuda.current_stream(dev).cuda_stream
    r = lib.dg_dev_build(ctypes.byref(d), row_ptr.data_ptr(), word.data_ptr(), w.data_ptr(), wt.data_ptr(),
                         wt_np.itemsize, cnt.data_ptr(), fill.data_ptr(), stream)
    if r != 0:
        raise RuntimeError(f"device generator failed (cuda error {r})")
    torch.cuda.current_stream(dev).synchronize()
    del cnt, fill
    return row_ptr, word, w


def device_csr_int8(tb: Tables, device="cuda"):
    """Device CSR with int8 weights and a power-of-two scale per row (w_acc =
    q << row_shift): (row_ptr, word, q8, row_shift).  Built from the int32
    (2^-16) weights of the same network, which are freed afterwards."""
    import torch

    row_ptr, word, w32 = device_csr(tb, "int32", device=device)
    q8 = torch.empty(w32.numel(), dtype=torch.int8, device=w32.device)
    rs = torch.empty(tb.n, dtype=torch.uint8, device=w32.device)
    stream = torch.cuda.current_stream(w32.device).cuda_stream
    r = _dev_lib().dg_dev_quantize_int8(row_ptr.data_ptr(), w32.data_ptr(), tb.n, q8.data_ptr(), rs.data_ptr(),
                                        stream)
    if r != 0:
        raise RuntimeError(f"int8 quantisation failed (cuda error {r})")
    torch.cuda.current_stream(w32.device).synchronize()
    del w32
    return row_ptr, word, q8, rs
