"""The seeded input generator: structure of the synthetic voxel networks and
agreement of its pull form (oracle input) with its outgoing CSR (GPU input)."""
import numpy as np
import pytest

from paper_2308_01241_gb300 import netgen as ng


def _small(name, n, nv, K):
    cfg = ng.load_config(name)
    return ng.make_tables(cfg, n_neurons=n, n_vox=nv, K=K)


@pytest.mark.parametrize("name,n,nv,K", [("c1_single_voxel_1k", None, None, None),
                                         ("c2_multi_voxel_1m", 20011, 12, 60),
                                         ("c3_large_20m", 30000, 40, 50)])
def test_structure_and_transpose(name, n, nv, K):
    tb = _small(name, n, nv, K)
    pre, cls, wbin = ng.host_pull(tb)
    vs = tb.voxel_start
    vox = np.searchsorted(vs, np.arange(tb.n), side="right") - 1
    assert vs[-1] == tb.n and np.all(np.diff(vs) >= 2)
    i = np.arange(tb.n)[:, None]
    assert np.all(pre != i)                                 # no self loops
    assert np.all((pre >= 0) & (pre < tb.n))
    loc = pre - vs[vox[pre]]
    assert np.array_equal(cls, (loc >= tb.nexc[vox[pre]]).astype(np.uint8))  # class = E/I of the source
    intra = vox[pre] == vox[i]
    assert np.all(intra[:, : tb.K_intra])
    if tb.nv > 1:
        assert np.all(~intra[:, tb.K_intra:])               # long-range inputs ...
        assert np.all(cls[:, tb.K_intra:] == 0)             # ... are excitatory
    assert np.all((tb.delay_vv >= 1) & (tb.delay_vv <= tb.d_max))
    assert np.all(np.diag(tb.delay_vv) == 1)
    # outgoing CSR holds exactly the pull-form entries, rows by source
    row_ptr, word, wb = ng.host_push(tb, (pre, cls, wbin))
    assert row_ptr[-1] == tb.n * tb.K
    src = np.repeat(np.arange(tb.n), np.diff(row_ptr))
    tgt = (word & 0x3FFFFFFF).astype(np.int64)
    a = np.lexsort((wbin.ravel(), cls.ravel(), np.repeat(np.arange(tb.n), tb.K), pre.ravel()))
    b = np.lexsort((wb, word >> 30, tgt, src))
    assert np.array_equal(pre.ravel()[a], src[b])
    assert np.array_equal(np.repeat(np.arange(tb.n), tb.K)[a], tgt[b])
    assert np.array_equal(cls.ravel()[a], (word >> 30)[b])
    assert np.array_equal(wbin.ravel()[a], wb[b])


def test_pull_rows_are_counter_based():
    tb = _small("c2_multi_voxel_1m", 20011, 12, 60)
    full = ng.host_pull(tb)
    part = ng.host_pull(tb, 7000, 7100)
    for f, p in zip(full, part):
        assert np.array_equal(f[7000:7100], p)


def test_dti_rows_normalised_and_sparse():
    tb = ng.make_tables(ng.load_config("c3_large_20m"))
    assert tb.nv == 2000 and tb.voxel_start[-1] == 20_000_000
    m = np.diff(tb.dti_ptr)
    assert np.all(m == round(0.1 * 1999))
    ends = tb.dti_cum[tb.dti_ptr[1:] - 1]
    assert np.all(ends == np.uint64(1 << 32))
    sizes = np.diff(tb.voxel_start)
    cv = sizes.std() / sizes.mean()
    assert 0.5 < cv < 1.2  # log-normal, sigma 0.8


def test_weight_tables():
    tb = _small("c1_single_voxel_1k", None, None, None)
    w16 = tb.wtable("int16")
    w32 = tb.wtable("int32")
    assert w16.dtype == np.int16 and w32.dtype == np.int32
    assert np.all(np.diff(w32) >= 0) and w16.min() >= 0
    assert abs(np.log(tb.w_float).mean() - (-1.0)) < 1e-3   # LogNormal(-1, 0.5) quantiles
    assert abs(np.log(tb.w_float).std() - 0.5) < 0.01
    np.testing.assert_allclose(w16 / 4096.0, tb.w_float, atol=0.5 / 4096.0)


def test_ensemble_networks_are_disjoint_blocks():
    """The merged ensemble network is block-diagonal: every synapse joins two
    neurons of the same member or target network, and the copies of a group
    share its voxel sizes."""
    tb, lay = ng.make_ensemble_tables(ng.load_config("c4_ensemble"), groups=2, members=3, vox_range=[4, 7],
                                      neuron_range=[3000, 6000])
    vs = tb.voxel_start
    net_of_vox = np.full(tb.nv, -1)
    k_net = 0
    for g in range(lay.groups):
        assert len(lay.net_vox[g]) == lay.members + 1
        sizes = None
        for first, count in lay.net_vox[g]:
            assert count == lay.group_vox[g]
            net_of_vox[first:first + count] = k_net
            k_net += 1
            s = np.diff(vs[first:first + count + 1])
            sizes = s if sizes is None else sizes
            np.testing.assert_array_equal(s, sizes)
    assert np.all(net_of_vox >= 0)
    pre, cls, wbin = ng.host_pull(tb)
    vox = np.searchsorted(vs, np.arange(tb.n), side="right") - 1
    net = net_of_vox[vox]
    assert pre.shape[0] == tb.n and pre.size > 0
    np.testing.assert_array_equal(net[pre], np.repeat(net[:, None], pre.shape[1], axis=1))


def test_generator_philox_known_answers(tmp_path):
    """The generator's own Philox4x32-10 (netgen_core.h, shared by its host
    and device builds) on the published known-answer vectors."""
    import os
    import shutil
    import subprocess

    from helpers import philox_kat

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    ctr, key, want = philox_kat()
    lines = ["#include <stdio.h>", '#include "netgen_core.h"', "int main(void) {", "  uint32_t o[4];"]
    for c, k in zip(ctr, key):
        args = ", ".join(f"{int(x)}u" for x in list(c) + list(k))
        lines.append(f'  dg_philox({args}, o); printf("%u %u %u %u\\n", o[0], o[1], o[2], o[3]);')
    lines += ["  return 0;", "}"]
    src = tmp_path / "kat.c"
    src.write_text("\n".join(lines) + "\n")
    inc = os.path.join(os.path.dirname(ng.__file__), "csrc")
    exe = tmp_path / "kat"
    r = subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.split()
    got = np.array([int(x) for x in out], np.uint64).astype(np.uint32).reshape(-1, 4)
    np.testing.assert_array_equal(got, want)
