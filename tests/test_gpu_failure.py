"""The device-side failure path, exercised without a fault.

The neuron update waits on its TMA stages with a bounded wait; when a wait
gives up the kernel records it and the call returns DTB_ETIMEOUT.  Here the
same wait runs on an mbarrier that nothing arrives at (so it must give up),
and on one that completes (so it must not); afterwards the context is still
usable and a network steps bit-exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01241_gb300 import netgen as ng

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports_timeout():
    from paper_2308_01241_gb300 import dtb

    assert dtb._lib.dtb_bounded_wait_test(1 << 20, 1) == dtb.DTB_OK
    assert dtb._lib.dtb_bounded_wait_test(1 << 20, 0) == dtb.DTB_ETIMEOUT
    assert b"gave up" in dtb._lib.dtb_last_error()
    assert dtb._lib.dtb_bounded_wait_test(0, 0) == dtb.DTB_EINVAL
    # the context is still usable
    tb = ng.make_tables(ng.load_config("c1_single_voxel_1k"))
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull))
    net.step(120)
    rids, roff = oracle.OracleNet(ng.oracle_inputs(tb, pull), "f32").run(120)
    ids, off = net.get_spikes()
    np.testing.assert_array_equal(ids, rids)
    np.testing.assert_array_equal(off, roff)


def test_binding_rejects_misshaped_host_buffers():
    """Host buffers the library would read or write past are refused before
    the call; the network is unchanged afterwards."""
    from paper_2308_01241_gb300 import dtb

    tb = ng.make_tables(ng.load_config("c1_single_voxel_1k"))
    pull = ng.host_pull(tb)
    net = dtb.from_tables(tb, dtb.host_csr(tb, pull))
    net.step(40)
    V, j, ref, ring, t = net.get_state()
    with pytest.raises(ValueError, match="V has shape"):
        net.set_state(V=V[:-1], t=t)
    with pytest.raises(ValueError, match="ring has shape"):
        net.set_state(ring=ring[:-1], t=t)
    with pytest.raises(ValueError, match="off_out"):
        net.get_spikes(off_out=np.zeros(10, np.int64))
    with pytest.raises(ValueError, match="ran 40 steps"):
        net.get_spikes(7)
    ids, off = net.get_spikes(40)
    assert off.shape == (41,) and off[-1] == ids.size
    V2, j2, ref2, ring2, t2 = net.get_state()
    assert t2 == t
    np.testing.assert_array_equal(V2, V)
    np.testing.assert_array_equal(ring2, ring)
