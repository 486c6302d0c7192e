"""The C-ABI boundary on the CPU: libdtb.so loads, exports every function
include/dtb.h declares, and rejects malformed descriptions with DTB_EINVAL
and a message before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dtb():
    from paper_2308_01241_gb300 import build

    build.build()
    from paper_2308_01241_gb300 import dtb as m

    return m


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"^\s*(?:dtb_status|const char\*|int)\s+(\w+)\(", txt, re.M)))


def test_every_declared_symbol_is_exported(dtb):
    names = _declared("dtb.h")
    assert len(names) >= 15
    lib = ctypes.CDLL(dtb.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_generator_library_exports(dtb):
    from paper_2308_01241_gb300 import netgen

    dev = ctypes.CDLL(netgen.DEV_LIB)
    host = ctypes.CDLL(netgen.build_host())
    names = _declared("dtbgen.h")
    assert "dg_dev_build" in names and "dg_host_pull" in names
    for n in names:
        assert hasattr(dev if n.startswith("dg_dev") else host, n), n


def _desc(dtb, **over):
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dt)
        keep.append(a)
        return a.ctypes.data

    d = dtb.dtb_network_desc()
    d.n_neurons, d.n_voxels, d.n_channels = 4, 1, 2
    d.voxel_start = arr([0, 4], np.int64)
    d.voxel_params = arr(np.ones(19), np.float64)
    d.dt, d.nu_ext, d.w_ext, d.weight_format, d.weight_shift, d.d_max = 0.1, 0.0, 65536, 1, 0, 1
    d.row_ptr = arr([0, 1, 1, 1, 1], np.int64)
    d.syn_word = arr([1], np.uint32)
    d.syn_w = arr([5], np.int32)
    d.delay_vv = arr([1], np.uint8)
    for k, v in over.items():
        if isinstance(v, tuple):
            setattr(d, k, arr(*v))
        else:
            setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over,msg", [
    (dict(n_neurons=0), "n_neurons"),
    (dict(n_channels=3), "n_channels"),
    (dict(voxel_start=([0, 3], np.int64)), "voxel_start"),
    (dict(delay_vv=([2], np.uint8)), "delay"),
    (dict(d_max=0), "d_max"),
    (dict(weight_format=7), "weight_format"),
    (dict(dt=0.0), "dt"),
    (dict(row_ptr=None), "NULL"),
    (dict(delivery_mode=3), "delivery_mode"),
    (dict(delivery_mode=2, bin_capacity=-1), "bin_capacity"),
    (dict(delivery_mode=1, event_queue_capacity=(1 << 32) - 1), "event_queue_capacity"),
    (dict(n_neurons=1 << 30), "n_neurons"),
    (dict(n_voxels=0), "n_voxels"),
    (dict(n_voxels=65536), "n_voxels"),
    (dict(weight_shift=25), "weight_shift"),
    (dict(nu_ext=-1.0), "nu_ext"),
    (dict(bold_every=-1), "bold_every"),
    (dict(d_max=256), "d_max"),
    (dict(n_voxels=2, voxel_start=([0, 5, 4], np.int64), delay_vv=([1, 1, 1, 1], np.uint8),
          voxel_params=(np.ones(38), np.float64)), "not ascending"),
    (dict(voxel_params=(np.r_[0.0, np.ones(18)], np.float64)), "C must be > 0"),
    (dict(voxel_params=(np.r_[np.ones(12), -1.0, np.ones(6)], np.float64)), "tau must be > 0"),
    (dict(ou_enable=1, ou_tau=0.0, ou_sigma=1.0), "OU drive"),
    (dict(ou_enable=1, ou_tau=5.0, ou_sigma=-1.0), "OU drive"),
    (dict(ou_enable=1, ou_tau=5.0, ou_sigma=1.0, ou_mu=float("nan")), "OU drive"),
])
def test_bad_descriptions_rejected(dtb, over, msg):
    d, keep = _desc(dtb, **over)
    h = ctypes.c_void_p(1234)
    r = dtb._lib.dtb_create_network(ctypes.byref(d), ctypes.byref(h))
    assert r == dtb.DTB_EINVAL
    assert h.value is None
    assert msg in dtb.dtb_last_error()


def test_null_arguments(dtb):
    lib = dtb._lib
    assert lib.dtb_create_network(None, None) == dtb.DTB_EINVAL
    assert lib.dtb_step(None, 1) == dtb.DTB_EINVAL
    assert lib.dtb_destroy(None) == dtb.DTB_EINVAL
    assert lib.dtb_get_state(None, None, None, None, None, None) == dtb.DTB_EINVAL


def _null_args(f):
    """NULL for every pointer argument, 0 for every number."""
    nums = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, ctypes.c_size_t)
    return [0 if a in nums else None for a in f.argtypes]


def test_every_handle_call_rejects_a_null_handle(dtb):
    """Each call that takes a network or MLP handle, or device arrays, returns
    DTB_EINVAL with a message for NULL ones, before any CUDA call."""
    from paper_2308_01241_gb300 import surrogate_mlp  # noqa: F401  (sets the MLP signatures)

    lib = dtb._lib
    skip = {"dtb_last_error", "dtb_bounded_wait_test", "dtb_philox_device"}
    names = [n for n in dtb._SIGS if n not in skip]
    names += ["dtb_mlp_create", "dtb_mlp_destroy", "dtb_mlp_forward", "dtb_mlp_gradients", "dtb_mlp_train_step",
              "dtb_mlp_get_params"]
    for name in names:
        f = getattr(lib, name)
        assert f(*_null_args(f)) == dtb.DTB_EINVAL, name
        assert dtb.dtb_last_error(), name
    assert len(names) >= 30
    # every function either header declares is exercised here or named as skipped
    declared = set(_declared("dtb.h")) | set(_declared("dtb_surrogate.h"))
    assert declared == set(names) | skip


def test_delivery_modes_named_in_the_binding(dtb):
    assert dtb.DELIVERY == {"ring": 0, "queue": 1, "bins": 2}
    txt = open(os.path.join(ROOT, "include", "dtb.h")).read()
    for name, v in (("DTB_DELIVER_RING", 0), ("DTB_DELIVER_QUEUE", 1), ("DTB_DELIVER_BINS", 2)):
        assert re.search(rf"{name}\s*=\s*{v}\b", txt), name


def test_header_is_c99_and_matches_the_binding_layout(dtb, tmp_path):
    """A C99 program compiled against include/dtb.h (and the other two
    headers) and linked to libdtb.so: the headers are valid C, the symbols
    resolve at link time, a call goes
    through, and every field of dtb_network_desc sits at the offset the
    ctypes binding uses (a mismatch would shift every later field)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in dtb.dtb_network_desc._fields_]
    efields = [f[0] for f in dtb.dtb_ensemble_desc._fields_]
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "dtb.h"', '#include "dtb_surrogate.h"', '#include "dtbgen.h"',
           "int main(void) {", '  printf("size %zu\\n", sizeof(dtb_network_desc));',
           '  printf("esize %zu\\n", sizeof(dtb_ensemble_desc));']
    src += [f'  printf("{f} %zu\\n", offsetof(dtb_network_desc, {f}));' for f in fields]
    src += [f'  printf("e.{f} %zu\\n", offsetof(dtb_ensemble_desc, {f}));' for f in efields]
    src += ["  dtb_net* h = (dtb_net*)1;",
            "  const int rc = (int)dtb_create_network(NULL, &h);",
            '  printf("create %d %d\\n", rc, h == NULL);',
            '  printf("error %s\\n", dtb_last_error());',
            "  return 0;", "}"]
    c = tmp_path / "abi.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(dtb.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c), "-o",
                        str(exe), "-L", libdir, "-ldtb", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    got = dict(ln.split(" ", 1) for ln in out.stdout.strip().splitlines())
    assert int(got["size"]) == ctypes.sizeof(dtb.dtb_network_desc)
    for f in fields:
        assert int(got[f]) == getattr(dtb.dtb_network_desc, f).offset, f
    assert int(got["esize"]) == ctypes.sizeof(dtb.dtb_ensemble_desc)
    for f in efields:
        assert int(got["e." + f]) == getattr(dtb.dtb_ensemble_desc, f).offset, f
    assert got["create"] == f"{dtb.DTB_EINVAL} 1"
    assert "desc is NULL" in got["error"]


def _prototypes(header):
    """{name: [parameter type, ...]} of the functions a header declares."""
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(?:dtb_status|const char\*|int)\s+(\w+)\(([^;]*?)\);", txt, re.M | re.S):
        params = [p.strip() for p in " ".join(m.group(2).split()).split(",") if p.strip()]
        out[m.group(1)] = [] if params == ["void"] else [re.sub(r"\s*\b\w+$", "", p) for p in params]
    return out


def _kind(ctype_param):
    """('ptr', 8) for pointers, (name, bytes) for scalars."""
    t = ctype_param.replace("const ", "").strip()
    if t.endswith("*"):
        return ("ptr", 8)
    return {"int64_t": ("int", 8), "uint64_t": ("int", 8), "int32_t": ("int", 4), "float": ("float", 4),
            "double": ("float", 8), "size_t": ("int", 8), "int": ("int", 4)}[t]


def test_binding_argtypes_match_the_prototypes(dtb):
    from paper_2308_01241_gb300 import surrogate_mlp  # noqa: F401  (sets the MLP signatures)

    protos = {**_prototypes("dtb.h"), **_prototypes("dtb_surrogate.h")}
    assert len(protos) >= 30
    for name, params in protos.items():
        f = getattr(dtb._lib, name)
        assert f.argtypes is not None, name
        want_res = ctypes.c_char_p if name == "dtb_last_error" else ctypes.c_int32
        assert f.restype is want_res or ctypes.sizeof(f.restype) == 4 and want_res is ctypes.c_int32, name
        assert len(f.argtypes) == len(params), name
        for k, (p, a) in enumerate(zip(params, f.argtypes)):
            kind = _kind(p)
            if a in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(a, type) and issubclass(a, ctypes._Pointer)):
                got = ("ptr", 8)
            elif a in (ctypes.c_float, ctypes.c_double):
                got = ("float", ctypes.sizeof(a))
            else:
                got = ("int", ctypes.sizeof(a))
            assert got == kind, f"{name} argument {k}: header {p!r}, binding {a}"


def test_generator_binding_matches_its_header_and_struct(tmp_path):
    """The generator's ABI: argtypes against include/dtbgen.h, and the ctypes
    DgNet against the C dg_net field by field (compiled with the C compiler)."""
    import shutil
    import subprocess

    from paper_2308_01241_gb300 import netgen

    libs = {"dg_host": netgen._host_lib(), "dg_dev": netgen._dev_lib()}
    protos = _prototypes("dtbgen.h")
    assert set(protos) == {"dg_host_pull", "dg_host_transpose", "dg_dev_build", "dg_dev_quantize_int8"}
    for name, params in protos.items():
        f = getattr(libs["dg_dev" if name.startswith("dg_dev") else "dg_host"], name)
        assert len(f.argtypes) == len(params), name
        for k, (p, a) in enumerate(zip(params, f.argtypes)):
            is_ptr = a is ctypes.c_void_p or (isinstance(a, type) and issubclass(a, ctypes._Pointer))
            got = ("ptr", 8) if is_ptr else ("int", ctypes.sizeof(a))
            assert got == _kind(p), f"{name} argument {k}: header {p!r}, binding {a}"
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in netgen.DgNet._fields_]
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "netgen_core.h"', "int main(void) {",
           '  printf("size %zu\\n", sizeof(dg_net));']
    src += [f'  printf("{f} %zu\\n", offsetof(dg_net, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    c = tmp_path / "dg.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "dg"
    inc = os.path.join(ROOT, "paper_2308_01241_gb300", "netgen", "csrc")
    r = subprocess.run([cc, "-std=c99", "-I", inc, str(c), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(ln.split(" ", 1) for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          timeout=60).stdout.strip().splitlines())
    assert int(got["size"]) == ctypes.sizeof(netgen.DgNet)
    for f in fields:
        assert int(got[f]) == getattr(netgen.DgNet, f).offset, f


def test_missing_library_fails_loudly():
    """Without libdtb.so the binding refuses to import: there is no CPU or
    library fallback for any step of the path."""
    import subprocess
    import sys

    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2308_01241_gb300.build as b\n"
            "b.LIB = '/nonexistent/libdtb.so'\n"
            "try:\n"
            "    import paper_2308_01241_gb300.dtb\n"
            "except ImportError as e:\n"
            "    print('refused:', e)\n"
            "else:\n"
            "    print('imported')\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("refused:") and "no CPU fallback" in r.stdout
