"""Pins of the oracle's random drive.

* Philox4x32-10 against the known-answer vectors published with Salmon et
  al. 2011 (tests/golden/philox4x32_10_kat.txt);
* Philox4x32-10 (Salmon et al. 2011) against cuRAND's host-side
  PHILOX4_32_10 generator, a library implementation run on the CPU: its block
  b = (y:x)*65536 + z of the stream under seed s is Philox({x, y, z, 0},
  key = (s_lo, s_hi)), which covers counter words 0-2 and both key words;
* the Poisson inversion thresholds against floor(2^32 * P(K <= m)) evaluated
  exactly with 60-digit arithmetic;
* the drawn counts against the Poisson(lambda) law (mean, variance, pmf).
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from helpers import philox_kat

CURAND = "/usr/local/cuda/lib64/libcurand.so"


def test_philox_known_answers():
    ctr, key, out = philox_kat()
    assert len(out) == 3
    for c, k, o in zip(ctr, key, out):
        np.testing.assert_array_equal(oracle.philox4x32_10(c, k), o)


def _curand_blocks(seed, first_block, n_blocks):
    lib = ctypes.CDLL(CURAND)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * n_blocks, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(n_blocks, 4)


@pytest.mark.skipif(not os.path.exists(CURAND), reason="cuRAND not installed")
@pytest.mark.parametrize("seed", [0, 2, 0x1234567890ABCDEF, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("x,y", [(0, 0), (7, 0), (0, 5), (0xFFFFFFFF, 0x3FFF)])
def test_philox_matches_curand_host(seed, x, y):
    z0 = 65530  # offsets are 64-bit: (y:x) * 65536 + z must stay below 2^62 blocks
    blocks = _curand_blocks(seed, ((y << 32) | x) * 65536 + z0, 6)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in range(6):
        assert np.array_equal(oracle.philox4x32_10([x, y, z0 + b, 0], key), blocks[b])


def _exact_thresholds(lam):
    mpmath = pytest.importorskip("mpmath")

    mpmath.mp.dps = 60
    lam = mpmath.mpf(lam)
    p = mpmath.e ** (-lam)
    F = p
    out = []
    m = 0
    while True:
        if m > 0:
            p = p * lam / m
            F = F + p
        x = int(mpmath.floor(F * mpmath.mpf(2) ** 32))
        if x >= 2 ** 32 - 1:
            return out
        out.append(x)
        m += 1


@pytest.mark.parametrize("lam", [0.2, 0.05, 0.4, 1.0, 2.5])
def test_poisson_thresholds_exact(lam):
    lam = (lam * 1000.0 * 0.1) / 1000.0 if lam == 0.2 else lam
    T = oracle.poisson_thresholds(lam)
    assert list(T) == _exact_thresholds(float(lam))


def test_poisson_drive_thresholds_of_config():
    lam = (2000.0 * 0.1) / 1000.0  # nu_ext = 2 kHz, dt = 0.1 ms
    assert list(oracle.poisson_thresholds(lam)) == _exact_thresholds(lam)


def test_poisson_counts_law():
    from scipy.stats import poisson

    lam = 0.2
    k = np.concatenate([oracle.drive_counts(2, lam, t, 0, 100000) for t in range(10)])
    assert abs(k.mean() - lam) < 4 * np.sqrt(lam / k.size)
    assert abs(k.var() - lam) < 0.01
    counts = np.bincount(k, minlength=5)[:4]
    expect = poisson.pmf(np.arange(4), lam) * k.size
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 16.3  # 3 dof, p = 0.001
    # independent across neurons and steps
    a = oracle.drive_counts(2, lam, 0, 0, 100000)
    b = oracle.drive_counts(2, lam, 1, 0, 100000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < 0.02


@pytest.mark.parametrize("k", [4, 8, 1024 + 4])
def test_index_base_slice_reproduces_the_full_network(k):
    """Every draw is counter-based on the global neuron index, so unconnected
    neurons k .. k+m-1 simulated alone with index_base = k (initial voltage,
    Poisson drive, OU current) match the same neurons of the full network.
    index_base must be a multiple of 4 (else the oracle refuses it)."""
    from helpers import custom_net, params_row

    n, m = k + 37, 37

    def net(count, base):
        d = custom_net(count, np.zeros((count, 0), np.int32), np.zeros((count, 0), np.uint8),
                       np.zeros((count, 0), np.int32), params_row(), nu_ext=2000.0, w_ext=3 * 65536, seed=5,
                       init_seed=6)
        d["index_base"] = base
        d.update(ou=dict(mu=0.1, sigma=0.05, tau=5.0))
        return oracle.OracleNet(d, "f32")

    with pytest.raises(ValueError, match="multiple of 4"):
        net(m, k + 1)
    full, part = net(n, 0), net(m, k)
    np.testing.assert_array_equal(part.get_state()[0], full.get_state()[0][k:])
    for _ in range(3):
        full.run(40)
        part.run(40)
        Vf, jf = full.get_state()[:2]
        Vp, jp = part.get_state()[:2]
        np.testing.assert_array_equal(Vp, Vf[k:])
        np.testing.assert_array_equal(jp, jf[:, k:])
        np.testing.assert_array_equal(part.get_ou(), full.get_ou()[k:])


def test_wrapper_structs_match_the_c_header(tmp_path):
    """The ctypes Desc and BoldParams of the oracle's wrapper against the C
    orc_desc and orc_bold_params, field by field (a misplaced field would make
    the oracle simulate another network without any error)."""
    import ctypes
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    here = os.path.dirname(oracle.__file__)
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "dtb_oracle.h"', "int main(void) {"]
    for cname, cls in (("orc_desc", oracle.Desc), ("orc_bold_params", oracle.BoldParams)):
        src.append(f'  printf("{cname}.size %zu\\n", sizeof({cname}));')
        src += [f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));' for f, _ in cls._fields_]
    src += ["  return 0;", "}"]
    c = tmp_path / "orc.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "orc"
    r = subprocess.run([cc, "-std=c99", "-I", here, str(c), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout
    got = dict(ln.split(" ", 1) for ln in out.strip().splitlines())
    for cname, cls in (("orc_desc", oracle.Desc), ("orc_bold_params", oracle.BoldParams)):
        assert int(got[f"{cname}.size"]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, f"{cname}.{f}"
