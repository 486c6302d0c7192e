"""Batched data-assimilation ensemble (hierarchical mesoscopic data assimilation, section V.E).

G groups of uneven size, each with M member networks and one hidden target
network of the same voxel structure, are merged into one block-diagonal
network. One graph-launched step advances every member and target:
neuron update, compaction, delivery, drain and BOLD each span all of them.

Parameters and observations:
- Each voxel has one parameter, the log gain on g_AMPA and g_NMDA. The
  members draw it from a log-normal prior; the targets hold a hidden draw
  from the same prior.
- Every TR (800 ms) the BOLD of every voxel is sampled. The targets' BOLD is
  the observation, and each column is one voxel of one group.

The assimilation cycle runs behind the C ABI (dtb_ensemble_create,
dtb_assimilate): per TR the network steps one TR, the members' predictions and
the targets' observations are gathered from the BOLD samples on the device, a
stochastic EnKF with perturbed observations updates the parameters, and the
new conductances go straight into the network's constants, with no host round
trip.  This module only marshals.  Launch shapes are picked by `dtb_autotune`
before the run.

    python -m paper_2308_01241_gb300.ensemble [--n-tr 200] [--groups 8 --members 8]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import dtb, netgen


class Ensemble:
    def __init__(self, cfg_name="c4_ensemble", groups=None, members=None, vox_range=None, neuron_range=None,
                 delivery="bins", device="cuda:0", autotune=True, tr_steps=None, log=print):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        cfg = netgen.load_config(cfg_name)
        self.cfg = cfg
        self.tb, self.lay = netgen.make_ensemble_tables(cfg, groups, members, vox_range, neuron_range)
        tb, lay = self.tb, self.lay
        self.tr_steps = int(tr_steps or cfg["enkf"]["tr_steps"])
        t0 = time.time()
        self.csr = netgen.device_csr(tb, cfg["wfmt"], device=device)
        self.base = tb.vparams(1.0)
        self.net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=self.base, delay_vv=tb.delay_vv,
                               d_max=tb.d_max, csr=self.csr, wfmt=cfg["wfmt"], wshift=4, n_ch=int(cfg["n_ch"]),
                               dt=float(cfg["dt"]), nu_ext=float(cfg["nu_ext"]), w_ext=int(cfg["w_ext"]),
                               seed=int(cfg["seeds"]["drive"]), init_seed=int(cfg["seeds"]["init"]),
                               bold=cfg["bold"], bold_every=self.tr_steps, delivery=delivery,
                               log_capacity=1 << 16, device=device)
        self.setup_s = time.time() - t0
        self.shapes = None
        if autotune:
            self.shapes = self.net.autotune(20)
            self.net.reset()
        log(f"ensemble: {tb.n} neurons, {tb.nv} voxels, {tb.n * tb.K:.3g} synapses, groups of "
            f"{lay.group_vox} voxels, {lay.members} members + 1 target each; setup {self.setup_s:.1f} s, "
            f"shapes {self.shapes}")
        # columns: every voxel of every group; members contiguous per column
        self.cols = []  # (group, local voxel)
        for g, V in enumerate(lay.group_vox):
            self.cols += [(g, v) for v in range(V)]
        C, M = len(self.cols), lay.members
        pr = cfg["prior"]
        rng = np.random.Generator(np.random.Philox(int(cfg["seeds"]["prior"])))
        self.theta = (pr["log_gain_mean"] + pr["log_gain_sd"] * rng.standard_normal((C, M))).astype(np.float32)
        self.theta_star = (pr["log_gain_mean"] + pr["log_gain_sd"] * rng.standard_normal(C)).astype(np.float32)
        self.rng = np.random.Generator(np.random.Philox(int(cfg["seeds"]["enkf"])))
        # voxel index (in the merged network) of column c in copy k
        self.vox_idx = np.zeros((C, M + 1), np.int64)
        c = 0
        for g, V in enumerate(lay.group_vox):
            for k, (o, _) in enumerate(lay.net_vox[g]):
                self.vox_idx[c:c + V, k] = o + np.arange(V)
            c += V
        self.apply()

    def apply(self):
        """Writes exp(theta) into g_AMPA and g_NMDA of every member voxel and exp(theta*) into the targets'."""
        gain = np.ones(self.tb.nv)
        M = self.lay.members
        gain[self.vox_idx[:, :M].ravel()] = np.exp(self.theta.astype(np.float64)).ravel()
        gain[self.vox_idx[:, M]] = np.exp(self.theta_star.astype(np.float64))
        g = self.base[:, 6:10].copy()
        g[:, 0] *= gain
        g[:, 1] *= gain
        self.net.set_hyperparams(g)

    def assimilation(self, obs_sd_rel: float, inflation: float) -> dtb.Assimilation:
        """The ensemble behind the C ABI: column c = voxel c of its group, members
        the group's member copies of that voxel, observed by the target copy."""
        M = self.lay.members
        return dtb.Assimilation(self.net, self.vox_idx[:, :M], self.theta, self.base[:, 6:10], self.tr_steps,
                                target_voxel=self.vox_idx[:, M], obs_sd_rel=obs_sd_rel, inflation=inflation,
                                seed=int(self.cfg["seeds"]["enkf"]))

    def run(self, n_tr: int, spinup_tr: int = 5, obs_sd_rel=None, inflation=None, log=print):
        """spinup_tr TRs without analysis, then n_tr assimilation cycles in one
        dtb_assimilate call.  history[0] is the prior, history[k] the state after
        the analysis of TR k (its bold_corr: the members' mean prediction against
        the observation at that TR, before the analysis)."""
        cfg = self.cfg["enkf"]
        obs_sd_rel = float(obs_sd_rel if obs_sd_rel is not None else cfg["obs_sd_rel"])
        inflation = float(inflation if inflation is not None else cfg["inflation"])
        self.apply()
        t0 = time.time()
        self.net.step(spinup_tr * self.tr_steps)
        t1 = time.time()
        asm = self.assimilation(obs_sd_rel, inflation)
        th0 = asm.theta()
        th, hx, y = asm.assimilate(n_tr)
        t2 = time.time()
        self.theta = asm.theta()
        asm.close()

        def row(tr, theta, corr):
            return {"tr": tr, "param_rmse": float(np.sqrt(np.mean((theta.mean(1) - self.theta_star) ** 2))),
                    "spread": float(theta.std(1, ddof=1).mean()), "bold_corr": corr}

        hist = [row(spinup_tr - 1, th0, float("nan"))]
        for k in range(n_tr):
            yk, mk = y[k].astype(np.float64), hx[k].mean(1).astype(np.float64)
            corr = float(np.corrcoef(mk, yk)[0, 1]) if np.std(yk) > 0 and np.std(mk) > 0 else float("nan")
            hist.append(row(spinup_tr + k, th[k], corr))
            if k % 10 == 0 or k == n_tr - 1:
                h = hist[-1]
                log(f"TR {h['tr']:4d}: parameter RMSE {h['param_rmse']:.4f}, spread {h['spread']:.4f}, "
                    f"BOLD corr {h['bold_corr']:.3f}")
        return {"history": hist, "spinup_s": t1 - t0, "cycle_s": t2 - t1,
                "prior_rmse": hist[0]["param_rmse"], "final_rmse": hist[-1]["param_rmse"],
                "final_bold_corr": hist[-1]["bold_corr"], "steps": (spinup_tr + n_tr) * self.tr_steps}

    def close(self):
        self.net.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c4_ensemble")
    ap.add_argument("--n-tr", type=int, default=None)
    ap.add_argument("--spinup-tr", type=int, default=5)
    ap.add_argument("--groups", type=int, default=None)
    ap.add_argument("--members", type=int, default=None)
    ap.add_argument("--delivery", default="bins", choices=["ring", "queue", "bins"])
    a = ap.parse_args()
    ens = Ensemble(a.config, groups=a.groups, members=a.members, delivery=a.delivery,
                   log=lambda *m: print(*m, file=sys.stderr, flush=True))
    n_tr = a.n_tr if a.n_tr is not None else int(ens.cfg["enkf"]["n_tr"])
    t0 = time.time()
    res = ens.run(n_tr, spinup_tr=a.spinup_tr, log=lambda *m: print(*m, file=sys.stderr, flush=True))
    res["wall_s"] = time.time() - t0
    res["neurons"], res["voxels"], res["synapses"] = ens.tb.n, ens.tb.nv, ens.tb.n * ens.tb.K
    res["group_voxels"], res["members"], res["shapes"] = ens.lay.group_vox, ens.lay.members, ens.shapes
    res["ms_per_step"] = 1000.0 * (res["spinup_s"] + res["cycle_s"]) / res["steps"]
    hist = res.pop("history")
    res["rmse_by_tr"] = [round(h["param_rmse"], 5) for h in hist]
    res["bold_corr_by_tr"] = [round(h["bold_corr"], 4) for h in hist]
    print(json.dumps(res), flush=True)
    ens.close()


if __name__ == "__main__":
    main()
