"""Builds the native libraries in-tree (no install step):

* ``_build/libdtb.so``          the step library (C ABI of ``include/dtb.h``), sm_103a
* ``_build/libdtbgen_dev.so``   the device side of the seeded network generator
* ``_build/libdtbgen_host.so``  the host side of the network generator (gcc)

nvcc flags: ``-gencode arch=compute_103a,code=sm_103a -lineinfo`` and
``--fmad=false`` (no fused multiply-add may change a rounding of the neuron
update; the kernels also use explicit round-to-nearest intrinsics).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdtb.so")
SOURCES = ["step_kernels.cu", "setup_kernels.cu", "standalone.cu", "standalone_noalloc.cu", "assimilate.cu",
           "mlp.cu", "dtb_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(ROOT, "include", h) for h in ("dtb.h", "dtb_surrogate.h")]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *NVCC_FLAGS, "-c", s, "-o", o])
    from .netgen import DEV_LIB, build_host, dev_build_cmd

    gen_src = [os.path.join(HERE, "netgen", "csrc", f) for f in ("netgen_dev.cu", "netgen_core.h")]
    if force or _stale(DEV_LIB, gen_src):
        jobs.extend(dev_build_cmd())
    with cf.ThreadPoolExecutor(max_workers=max(1, min(4, os.cpu_count() or 1))) as ex:
        list(ex.map(_run, jobs))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    build_host(force)
    if verbose:
        print("built", LIB)
    return LIB


def ptxas_report() -> str:
    """Registers / spills / shared memory of every kernel (ptxas -v)."""
    out = []
    for src in SOURCES:
        r = subprocess.run([nvcc(), *ARCH, *NVCC_FLAGS, "-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o",
                            os.devnull], capture_output=True, text=True)
        out.append(r.stderr)
    return "\n".join(out)
