"""The batched assimilation ensemble on the GPU.

* the merged block-diagonal network (members + targets of uneven size)
  matches the oracle bit for bit, like any other network;
* dtb_autotune changes launch shapes only: after a reset the raster is the
  same as a fresh network's;
* a short assimilation (EnKF each TR on the targets' BOLD) moves the
  members' log gains toward the hidden ones.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01241_gb300 import netgen as ng

pytestmark = pytest.mark.gpu


def _small():
    cfg = ng.load_config("c4_ensemble")
    return cfg, *ng.make_ensemble_tables(cfg, groups=2, members=4, vox_range=[6, 10], neuron_range=[4000, 9000])


@pytest.mark.parametrize("delivery", ["ring", "queue", "bins"])
def test_merged_ensemble_network_bit_exact(delivery):
    from paper_2308_01241_gb300 import dtb

    cfg, tb, lay = _small()
    pull = ng.host_pull(tb)
    d = ng.oracle_inputs(tb, pull)
    rng = np.random.default_rng(0)
    d["vparams"][:, 6:8] *= np.exp(0.18 + 0.08 * rng.standard_normal(tb.nv))[:, None]
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=d["vparams"], delay_vv=tb.delay_vv,
                      d_max=tb.d_max, csr=dtb.host_csr(tb, pull), wfmt="int16", wshift=4, dt=d["dt"],
                      nu_ext=d["nu_ext"], w_ext=d["w_ext"], seed=d["seed"], init_seed=d["init_seed"],
                      bold=d["bold"], delivery=delivery)
    ref = oracle.OracleNet(d, "f32")
    net.step(300)
    ids, off = net.get_spikes()
    rids, roff = ref.run(300)
    np.testing.assert_array_equal(off, roff)
    np.testing.assert_array_equal(ids, rids)
    assert len(ids) > 500
    V = net.get_state()[0]
    np.testing.assert_array_equal(V, ref.get_state()[0])
    # autotune only changes launch shapes
    shapes = net.autotune(5)
    assert shapes["update_stages"] in (2, 3, 4)
    net.reset()
    net.step(300)
    np.testing.assert_array_equal(net.get_spikes()[0], rids)


def test_short_assimilation_reduces_parameter_error():
    from paper_2308_01241_gb300.ensemble import Ensemble

    # real 800 ms TRs: the BOLD response needs seconds to reflect the gains
    ens = Ensemble("c4_ensemble", groups=2, members=8, vox_range=[20, 30], neuron_range=[40000, 60000],
                   autotune=False, log=lambda *a: None)
    res = ens.run(15, spinup_tr=5, log=lambda *a: None)
    ens.close()
    rmse = [round(h["param_rmse"], 4) for h in res["history"]]
    corr = [round(h["bold_corr"], 3) for h in res["history"]]
    assert np.isfinite(res["final_bold_corr"]), corr
    # the mean over the last five TRs: single-TR values fluctuate with the perturbed observations
    assert np.mean(rmse[-5:]) < 0.8 * res["prior_rmse"], (rmse, corr)


def _perturbations(C, M, tr, seed):
    """The cycle's observation perturbations regenerated on the host: the
    Irwin-Hall(4) normal of the oracle's Philox4x32-10 at counter {m, c, TR, 4}."""
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    scale = np.float32(1.7320508075688772 / 4294967296.0)
    eps = np.zeros((C, M), np.float32)
    for c in range(C):
        for m in range(M):
            r = oracle.philox4x32_10(np.array([m, c, tr, 4], np.uint32), key)
            eps[c, m] = np.float32(np.float32(int(r.astype(np.int64).sum()) - (1 << 33)) * scale)
    return eps


def test_assimilation_cycle_on_the_device():
    """dtb_assimilate through the C ABI on a small merged ensemble (2 groups of
    4 members + 1 target), 3 TRs of 80 ms:
    * the gathered predictions and observations of the last TR are the BOLD
      samples of the member and target voxels, exactly;
    * each TR's analysis equals the FP64 oracle's EnKF on the same
      predictions, observations and perturbations (regenerated on the host
      from the oracle's Philox), within FP32 rounding: |d| <= 1e-4 (1 + |theta|);
    * the re-sampled constants are those dtb_set_hyperparams derives from
      g_base * exp(theta): from one checkpoint, the network after the cycle and
      the network given those conductances by the host produce the same raster."""
    from paper_2308_01241_gb300 import dtb

    cfg, tb, lay = _small()
    M, T, seed, infl, sd_rel = lay.members, 800, 16, 1.03, 0.02
    base = tb.vparams(1.0)
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=base, delay_vv=tb.delay_vv, d_max=tb.d_max,
                      csr=dtb.host_csr(tb, ng.host_pull(tb)), wfmt="int16", wshift=4, dt=float(cfg["dt"]),
                      nu_ext=float(cfg["nu_ext"]), w_ext=int(cfg["w_ext"]), seed=12, init_seed=13, bold=cfg["bold"],
                      bold_every=T, delivery="bins")
    member, target = [], []
    for g, V in enumerate(lay.group_vox):
        copies = lay.net_vox[g]
        for v in range(V):
            member.append([copies[k][0] + v for k in range(M)])
            target.append(copies[M][0] + v)
    member, target = np.array(member, np.int32), np.array(target, np.int32)
    C = len(target)
    rng = np.random.default_rng(3)
    theta0 = (0.18 + 0.08 * rng.standard_normal((C, M))).astype(np.float32)
    theta_star = 0.18 + 0.08 * rng.standard_normal(C)
    g = base[:, 6:10].copy()
    g[target, 0] *= np.exp(theta_star)
    g[target, 1] *= np.exp(theta_star)
    net.set_hyperparams(g)
    asm = dtb.Assimilation(net, member, theta0, base[:, 6:10], T, target_voxel=target, obs_sd_rel=sd_rel,
                           inflation=infl, seed=seed)
    np.testing.assert_array_equal(asm.theta(), theta0)
    net.step(2 * T)
    n_tr = 3
    th, hx, y = asm.assimilate(n_tr)
    ys = net.get_bold_samples()[-1]
    np.testing.assert_array_equal(hx[-1], ys[member])
    np.testing.assert_array_equal(y[-1], ys[target])
    prev = theta0.astype(np.float64)
    for k in range(n_tr):
        sd = (np.float32(sd_rel) * np.maximum(np.abs(y[k]), np.float32(1e-4))).astype(np.float64)
        want = oracle.enkf(prev, hx[k], y[k], sd, _perturbations(C, M, k, seed), lam=infl)
        got = th[k].astype(np.float64)
        assert np.all(np.abs(got - want) <= 1e-4 * (1 + np.abs(want))), k
        prev = got
    assert np.abs(th[-1] - theta0).max() > 1e-3  # the cycle moved the parameters
    np.testing.assert_array_equal(asm.theta(), th[-1])
    # re-sampled constants == host-derived constants: same raster from one checkpoint
    blob = net.save_state()
    net.step(400)
    ids_dev = net.get_spikes()[0].copy()
    net.load_state(blob)
    g2 = g.copy()
    gain = np.exp(th[-1].astype(np.float64))
    g2[member.ravel(), 0] = base[member.ravel(), 6] * gain.ravel()
    g2[member.ravel(), 1] = base[member.ravel(), 7] * gain.ravel()
    net.set_hyperparams(g2)
    net.step(400)
    np.testing.assert_array_equal(net.get_spikes()[0], ids_dev)
    assert len(ids_dev) > 100
    asm.close()
    net.close()


def test_assimilation_with_host_observations_and_bad_arguments():
    """bold_obs given by the caller replaces the target voxels; the call and
    the ensemble's creation reject bad arguments with DTB_EINVAL / DTB_ESTATE."""
    from paper_2308_01241_gb300 import dtb

    cfg, tb, lay = _small()
    base = tb.vparams(1.0)
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=base, delay_vv=tb.delay_vv, d_max=tb.d_max,
                      csr=dtb.host_csr(tb, ng.host_pull(tb)), wfmt="int16", wshift=4, bold=cfg["bold"],
                      bold_every=400, delivery="queue")
    member = np.arange(8, dtype=np.int32).reshape(2, 4)
    theta0 = np.full((2, 4), 0.1, np.float32)
    with pytest.raises(dtb.DtbError, match="tr_steps"):
        dtb.Assimilation(net, member, theta0, base[:, 6:10], 500)
    with pytest.raises(dtb.DtbError, match="twice"):
        dtb.Assimilation(net, np.zeros((2, 4), np.int32), theta0, base[:, 6:10], 400)
    with pytest.raises(dtb.DtbError, match="member voxel"):
        dtb.Assimilation(net, member + tb.nv, theta0, base[:, 6:10], 400)
    asm = dtb.Assimilation(net, member, theta0, base[:, 6:10], 400, inflation=1.0)
    with pytest.raises(dtb.DtbError, match="target"):
        asm.assimilate(1)  # no observations and no target voxels
    obs = np.array([[0.01, -0.02], [0.015, 0.0]], np.float32)
    th, hx, y = asm.assimilate(2, bold_obs=obs)
    np.testing.assert_array_equal(y, obs)
    net.step(7)
    with pytest.raises(dtb.DtbError) as e:
        asm.assimilate(1, bold_obs=obs[:1])
    assert e.value.code == dtb.DTB_ESTATE
    asm.close()
    net.close()
