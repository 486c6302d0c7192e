"""Small network builders shared by the tests (inputs only, no method arithmetic)."""
from __future__ import annotations

import os

import numpy as np

BOLD = dict(eps=0.02, tau_s=0.8, tau_f=0.4, tau_0=1.0, alpha=0.32, E0=0.34, V0=0.02)


def params_row(C=0.5, gL=0.025, EL=-70.0, Vth=-50.0, Vreset=-55.0, t_ref=2.0,
               g=(0.002, 0.00002, 0.01, 0.0005), tau=(2.0, 100.0, 6.0, 100.0),
               E=(0.0, 0.0, -70.0, -100.0), I_ext=0.0) -> np.ndarray:
    row = np.zeros(19, np.float64)
    row[0:6] = (C, gL, EL, Vth, Vreset, t_ref)
    row[6:10] = g
    row[10:14] = tau
    row[14:18] = E
    row[18] = I_ext
    return row


def custom_net(n, pre, cls, w, vparams, voxel_start=None, delay_vv=None, d_max=1, n_ch=2,
               nu_ext=0.0, w_ext=65536, wfmt=1, wshift=0, dt=0.1, seed=2, init_seed=3) -> dict:
    """Oracle input dict for an explicit pull-form network."""
    pre = np.asarray(pre, np.int32).reshape(n, -1)
    K = pre.shape[1]
    if voxel_start is None:
        voxel_start = np.array([0, n], np.int64)
    nv = len(voxel_start) - 1
    if delay_vv is None:
        delay_vv = np.ones((nv, nv), np.uint8)
    vparams = np.asarray(vparams, np.float64).reshape(-1, 19)
    if vparams.shape[0] == 1 and nv > 1:
        vparams = np.tile(vparams, (nv, 1))
    return dict(n=n, n_vox=nv, n_ch=n_ch, voxel_start=np.asarray(voxel_start, np.int64), vparams=vparams,
                dt=dt, nu_ext=nu_ext, w_ext=w_ext, K=K, pre=pre, cls=np.asarray(cls, np.uint8).reshape(n, K),
                wfmt=wfmt, w=np.asarray(w).reshape(n, K), wshift=wshift, delay_vv=np.asarray(delay_vv, np.uint8),
                d_max=d_max, seed=seed, init_seed=init_seed, bold=dict(BOLD))


def lone_neurons(n=4, **prm) -> dict:
    """n unconnected neurons (K = 0) in one voxel, no drive."""
    return custom_net(n, np.zeros((n, 0), np.int32), np.zeros((n, 0), np.uint8), np.zeros((n, 0), np.int32),
                      params_row(**prm))


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def philox_kat():
    """(ctr [m][4], key [m][2], out [m][4]) uint32 of the published Philox4x32-10
    known answers in golden/philox4x32_10_kat.txt."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                rows.append([int(x, 16) for x in line])
    a = np.array(rows, np.uint64).astype(np.uint32)
    assert a.shape[1] == 10
    return a[:, 0:4], a[:, 4:6], a[:, 6:10]


# ----------------------------------------------------------------------------- digests
# Byte layouts hashed identically by the golden-value scripts (oracle side)
# and by the GPU tests (library side): plain serialisation, no method arithmetic.
def table_digest(tb, gain: float) -> str:
    """sha256 of a network's voxel-level input tables and its parameter rows
    at the given gain (the synapses are integer functions of these and the seed)."""
    import hashlib

    h = hashlib.sha256()
    for a in (tb.voxel_start, tb.nexc, tb.dti_ptr, tb.dti_src, tb.dti_cum, tb.delay_vv, tb.wtable("int32"),
              tb.vparams(gain)):
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode() + str(a.shape).encode())
        h.update(a.tobytes())
    h.update(repr(tb.key).encode())
    return h.hexdigest()


def raster_digest(ids, off) -> str:
    """sha256 of a raster chunk: the per-step counts (int64) then the ids (int32)."""
    import hashlib

    off = np.asarray(off, np.int64)
    h = hashlib.sha256()
    h.update(np.diff(off).astype("<i8").tobytes())
    h.update(np.asarray(ids[off[0]:off[-1]], "<i4").tobytes())
    return h.hexdigest()


def array_digest(a) -> str:
    import hashlib

    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.astype(a.dtype.newbyteorder("<")).tobytes()).hexdigest()


def read_golden(name: str) -> dict:
    """Key/value lines of a golden file: 'key value ...' (comments after #)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out[line[0]] = line[1:]
    return out
