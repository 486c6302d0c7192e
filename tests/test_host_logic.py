"""Host-side logic of the package's drivers, on the CPU: the surrogate MLP's
flat parameter layout (as include/dtb_surrogate.h states it), the afferent
rates and the row-normalised voxel coupling the surrogate's features use, and
the precision study's rate and BOLD comparison."""
import numpy as np
import pytest

from paper_2308_01241_gb300 import netgen as ng


def test_mlp_parameter_layout_round_trips():
    from paper_2308_01241_gb300.surrogate_mlp import flatten, unflatten

    n_in, width, depth, n_out = 5, 7, 3, 2
    rng = np.random.default_rng(0)
    sizes = [n_in] + [width] * depth + [n_out]
    params = [(rng.standard_normal((a, b)).astype(np.float32), rng.standard_normal(b).astype(np.float32))
              for a, b in zip(sizes[:-1], sizes[1:])]
    flat = flatten(params)
    assert flat.dtype == np.float32
    assert flat.size == sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    # W_0 [n_in][width] row-major, then b_0, then W_1 ...
    np.testing.assert_array_equal(flat[:n_in * width], params[0][0].ravel())
    np.testing.assert_array_equal(flat[n_in * width:n_in * width + width], params[0][1])
    back = unflatten(flat, n_in, width, depth, n_out)
    for (W, b), (W2, b2) in zip(params, back):
        np.testing.assert_array_equal(W, W2)
        np.testing.assert_array_equal(b, b2)


def _coupling_tables():
    return ng.make_tables(ng.load_config("c2_multi_voxel_1m"), n_neurons=20000, n_vox=12, K=40)


def test_voxel_coupling_rows_are_normalised():
    from paper_2308_01241_gb300.surrogate import dti_matrix

    tb = _coupling_tables()
    rows, cols, vals = dti_matrix(tb)
    assert np.all(vals >= 0) and np.all(cols != rows)  # no self coupling
    sums = np.bincount(rows, weights=vals, minlength=tb.nv)
    has = np.diff(tb.dti_ptr) > 0
    assert has.any()
    np.testing.assert_allclose(sums[has], 1.0, atol=1e-9)
    assert np.all(sums[~has] == 0)


def test_afferent_rate_is_the_coupling_matrix_product():
    from paper_2308_01241_gb300.surrogate import afferent, dti_matrix

    tb = _coupling_tables()
    P = dti_matrix(tb)
    rates = np.random.default_rng(1).uniform(0, 30, tb.nv)
    dense = np.zeros((tb.nv, tb.nv))
    np.add.at(dense, (P[0], P[1]), P[2])
    np.testing.assert_allclose(afferent(rates, P), dense @ rates, rtol=1e-12)


def test_precision_comparison_metrics():
    from paper_2308_01241_gb300.precision import _compare

    rng = np.random.default_rng(2)
    rate = np.r_[rng.uniform(2, 20, 50), np.zeros(5), [0.5]]  # 6 voxels below 1 Hz are left out
    bold = rng.standard_normal((40, rate.size))
    ref = {7: {"rate": rate, "bold": bold, "ms_per_step": 0.3}}
    same = _compare(ref, {7: {"rate": rate.copy(), "bold": bold.copy(), "ms_per_step": 0.2}})[7]
    assert same["rate_dev_max"] == 0 and same["frac_voxels_within_2pct"] == 1.0
    assert same["voxels_active"] == 50 and same["bold_pearson"] == pytest.approx(1.0)
    var_rate = rate.copy()
    var_rate[:10] *= 1.05  # ten active voxels 5 % off
    off = _compare(ref, {7: {"rate": var_rate, "bold": bold, "ms_per_step": 0.2}})[7]
    assert off["rate_dev_max"] == pytest.approx(0.05) and off["frac_voxels_within_2pct"] == pytest.approx(0.8)


class _FakeSpikeLib:
    """Stands in for libdtb's dtb_get_spikes: a call of `steps` steps whose
    raster is `ids`; writes step_offsets [steps + 1] and the ids as the C
    function does, and records the capacities it was given."""

    def __init__(self, steps, ids):
        import ctypes

        self.ctypes = ctypes
        self.steps, self.ids, self.calls = steps, np.asarray(ids, np.int32), []

    def dtb_get_spikes(self, h, off_p, ids_p, cap, n_out_ref):
        c = self.ctypes
        total = self.ids.size
        n_out_ref._obj.value = total  # the binding passes ctypes.byref(c_int64)
        self.calls.append((off_p, ids_p, cap))
        if off_p:
            off = np.linspace(0, total, self.steps + 1).astype(np.int64)
            c.memmove(off_p, off.ctypes.data, off.nbytes)
        if ids_p and cap >= total:
            c.memmove(ids_p, self.ids.ctypes.data, self.ids.nbytes)
        return 0


def _fake_network(monkeypatch, steps, ids):
    from paper_2308_01241_gb300 import dtb

    fake = _FakeSpikeLib(steps, ids)
    monkeypatch.setattr(dtb, "_lib", fake)
    net = object.__new__(dtb.Network)
    net.h, net._nsteps = 1, steps
    return net, fake


def test_get_spikes_into_preallocated_buffers(monkeypatch):
    """The bench's end-to-end read: the raster of a c-step call into a slice
    of a larger offsets buffer and an ids buffer with spare room."""
    ids = np.arange(7, 7 + 90, dtype=np.int32)
    net, fake = _fake_network(monkeypatch, 250, ids)
    ids_buf = np.zeros(1 << 12, np.int32)
    off_buf = np.zeros(251, np.int64)
    got_ids, got_off = net.get_spikes(250, ids_out=ids_buf, off_out=off_buf[:251])
    np.testing.assert_array_equal(got_ids, ids)
    assert got_off.shape == (251,) and got_off[-1] == 90 and got_off[0] == 0
    assert np.shares_memory(got_ids, ids_buf) and np.shares_memory(got_off, off_buf)
    assert fake.calls[-1][2] == ids_buf.size
    # a shorter last chunk reuses the front of the same buffers
    net._nsteps = fake.steps = 37
    got_ids, got_off = net.get_spikes(37, ids_out=ids_buf, off_out=off_buf[:38])
    assert got_off.shape == (38,) and got_off[-1] == 90
    # an ids buffer too small for the raster is replaced, not overrun
    small = np.zeros(10, np.int32)
    got_ids, _ = net.get_spikes(ids_out=small)
    assert not np.shares_memory(got_ids, small)
    np.testing.assert_array_equal(got_ids, ids)
