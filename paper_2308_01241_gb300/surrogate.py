"""Learned surrogate of a voxel over one assimilation window, and surrogate-driven assimilation.

The surrogate is an MLP, 12 -> 256 -> 256 -> 256 -> 6 with GELU, trained by
the library's BF16 tensor-core kernels (include/dtb_surrogate.h). It maps
what a voxel knows at the start of a window (TR = 800 ms) to what the
simulator produces during it.

Inputs (12):
- the voxel's 4 receptor hyper-parameters: the log gains on g_AMPA, g_NMDA,
  g_GABAa, g_GABAb;
- 8 summaries of the previous window: its own rate, the four Balloon
  states s, f, v, q, the DTI-weighted rate of its source voxels, its
  previous AMPA log gain, and the log of its size.

Outputs (6): the window's rate, the BOLD signal y at its end, and the four
Balloon states. The paper's data assimilation (section V.E) runs the
spiking model for every ensemble member; here the MLP replaces it in the
predict step.

Three phases (one command):

1. **Data.** The simulator runs the merged ensemble network (all networks of
   the batched ensemble config). The hyper-parameters of every voxel follow
   an AR(1) walk across windows around the prior (correlation 0.8 per
   window, the prior's spread as stationary spread), so the previous
   window's state is informative as it is during assimilation, where the
   EnKF moves the parameters a little per TR. Every window records one
   (input, output) row per voxel.
2. **Training.** Inputs and targets are standardised with the training
   rows' mean and standard deviation; Adam on mini-batches, on the GPU. The
   report gives the validation R^2 of each output.
3. **Assimilation.** The surrogate drives an ensemble of 1,024 members
   (8 groups x 128). The simulator still runs the 8 hidden targets and 8
   audit members per group (6 %). Every TR, the surrogate's rate prediction
   for the audit members is compared with their simulated rate; if the mean
   relative error exceeds 5 %, that TR's analysis falls back to the
   simulated members (the plain simulator). The audit members are the first
   8 surrogate members of each group (same parameter draws), and the
   surrogate's BOLD error on them (a running mean square) is added to the
   observation noise of the surrogate-driven analysis. The report compares the
   recovered hyper-parameters and the BOLD with the simulator-driven run of
   the same groups and targets, and the cost per TR with the cost the
   simulator would have for 1,024 members.

    python -m paper_2308_01241_gb300.surrogate [--windows 150] [--n-tr 40]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import dtb, netgen
from .ensemble import Ensemble
from .surrogate_mlp import MLP

N_IN, WIDTH, DEPTH, N_OUT = 12, 256, 3, 6
R_SCALE = 20.0    # Hz
S_SCALE = 100.0   # Balloon states and BOLD around rest


def _log(*m):
    print(*m, file=sys.stderr, flush=True)


def dti_matrix(tb, lay):
    """Row-normalised inter-voxel coupling P[v, u] of the merged network (sparse as dense rows per voxel)."""
    rows, cols, vals = [], [], []
    for v in range(tb.nv):
        a, b = tb.dti_ptr[v], tb.dti_ptr[v + 1]
        if b == a:
            continue
        cum = tb.dti_cum[a:b].astype(np.float64) / 2.0 ** 32
        p = np.diff(np.concatenate([[0.0], cum]))
        rows += [v] * (b - a)
        cols += list(tb.dti_src[a:b])
        vals += list(p)
    return np.array(rows), np.array(cols), np.array(vals)


def afferent(rates, P):
    rows, cols, vals = P
    out = np.zeros_like(rates)
    np.add.at(out, rows, vals * rates[cols])
    return out


def features(theta4, r_prev, bold_state, aff, th_prev, logn):
    """[V][12] inputs (normalised)."""
    s, f, v, q = bold_state
    return np.column_stack([theta4, r_prev / R_SCALE, s * S_SCALE, (f - 1) * S_SCALE, (v - 1) * S_SCALE,
                            (q - 1) * S_SCALE, aff / R_SCALE, th_prev, logn]).astype(np.float32)


def targets(rate, y, bold_state):
    s, f, v, q = bold_state
    return np.column_stack([rate / R_SCALE, y * S_SCALE, s * S_SCALE, (f - 1) * S_SCALE, (v - 1) * S_SCALE,
                            (q - 1) * S_SCALE]).astype(np.float32)


def generate(n_windows, log=_log):
    """Simulator windows on the merged ensemble network with random hyper-parameters per window."""
    cfg = netgen.load_config("c4_ensemble")
    tb, lay = netgen.make_ensemble_tables(cfg)
    csr = netgen.device_csr(tb, cfg["wfmt"])
    base = tb.vparams(1.0)
    tr = int(cfg["enkf"]["tr_steps"])
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=base, delay_vv=tb.delay_vv, d_max=tb.d_max,
                      csr=csr, wfmt=cfg["wfmt"], wshift=4, dt=float(cfg["dt"]), nu_ext=float(cfg["nu_ext"]),
                      w_ext=int(cfg["w_ext"]), seed=int(cfg["seeds"]["drive"]) + 7,
                      init_seed=int(cfg["seeds"]["init"]), bold=cfg["bold"], bold_every=tr, delivery="queue",
                      log_capacity=1 << 16)
    rng = np.random.default_rng(2024)
    sizes = np.diff(tb.voxel_start).astype(np.float64)
    logn = np.log(sizes) - 9.0
    P = dti_matrix(tb, lay)
    dt_s = float(cfg["dt"]) * 1e-3
    X, Y = [], []
    prev = None
    t0 = time.time()
    rho = 0.8
    mean4 = np.array([0.18, 0.18, 0.0, 0.0])
    sd4 = np.array([0.12, 0.12, 0.05, 0.05])
    th4 = mean4 + sd4 * rng.standard_normal((tb.nv, 4))
    for w in range(n_windows + 1):
        th4 = mean4 + rho * (th4 - mean4) + np.sqrt(1 - rho * rho) * sd4 * rng.standard_normal((tb.nv, 4))
        th4[:, 1] = th4[:, 0] + 0.02 * rng.standard_normal(tb.nv)
        thA = th4[:, 0].copy()
        g = base[:, 6:10] * np.exp(th4)
        net.set_hyperparams(g)
        c0 = net.voxel_spikes()
        net.step(tr)
        rate = (net.voxel_spikes() - c0) / (sizes * tr * dt_s)
        y, st = net.get_bold()
        st = st.astype(np.float64)
        if prev is not None:
            r_prev, st_prev, thA_prev = prev
            X.append(features(th4, r_prev, st_prev, afferent(r_prev, P), thA_prev, logn))
            Y.append(targets(rate, y.astype(np.float64), st))
        prev = (rate, st, thA)
        if w % 20 == 0:
            log(f"window {w}: {time.time() - t0:.1f} s, mean rate {rate.mean():.2f} Hz")
    net.close()
    return np.concatenate(X), np.concatenate(Y), time.time() - t0


class Surrogate:
    """The trained MLP with its input and target standardisation."""

    def __init__(self, mlp, x_mu, x_sd, y_mu, y_sd):
        import torch

        self.mlp = mlp
        f = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()  # noqa: E731
        self.x_mu, self.x_sd, self.y_mu, self.y_sd = f(x_mu), f(x_sd), f(y_mu), f(y_sd)

    def predict(self, x):
        """x [B][N_IN] float32 device tensor (raw features) -> [B][N_OUT] raw targets."""
        import torch

        xs = ((x - self.x_mu) / self.x_sd).contiguous()
        y = torch.empty((x.shape[0], N_OUT), dtype=torch.float32, device=x.device)
        self.mlp.forward(xs, y)
        return y * self.y_sd + self.y_mu

    def close(self):
        self.mlp.close()

    def save(self, path):
        flat = {f"W{i}": W for i, (W, _) in enumerate(self.mlp.params())}
        flat.update({f"b{i}": b for i, (_, b) in enumerate(self.mlp.params())})
        np.savez(path, x_mu=self.x_mu.cpu().numpy(), x_sd=self.x_sd.cpu().numpy(),
                 y_mu=self.y_mu.cpu().numpy(), y_sd=self.y_sd.cpu().numpy(), **flat)

    @staticmethod
    def load(path, max_batch=1 << 17):
        z = np.load(path)
        params = [(z[f"W{i}"], z[f"b{i}"]) for i in range(DEPTH + 1)]
        mlp = MLP(params, N_IN, WIDTH, DEPTH, N_OUT, max_batch=max_batch)
        return Surrogate(mlp, z["x_mu"], z["x_sd"], z["y_mu"], z["y_sd"])


def train(X, Y, epochs=8, batch=4096, lr=1e-3, log=_log, max_batch=1 << 17):
    import torch

    rng = np.random.default_rng(7)
    sizes = [N_IN] + [WIDTH] * DEPTH + [N_OUT]
    params = [(rng.standard_normal((sizes[i], sizes[i + 1])) * np.sqrt(2.0 / sizes[i]), np.zeros(sizes[i + 1]))
              for i in range(len(sizes) - 1)]
    n = X.shape[0]
    perm = rng.permutation(n)
    n_val = n // 20
    val, tr_idx = perm[:n_val], perm[n_val:]
    x_mu, x_sd = X[tr_idx].mean(0), X[tr_idx].std(0) + 1e-6
    y_mu, y_sd = Y[tr_idx].mean(0), Y[tr_idx].std(0) + 1e-6
    dX = torch.from_numpy(((X - x_mu) / x_sd).astype(np.float32)).cuda()
    dY = torch.from_numpy(((Y - y_mu) / y_sd).astype(np.float32)).cuda()
    net = MLP(params, N_IN, WIDTH, DEPTH, N_OUT, max_batch=max(batch, max_batch))
    t0 = time.time()
    hist = []
    vi = torch.from_numpy(val[:65536]).cuda()
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(tr_idx)).cuda()
        losses = []
        for k in range(0, order.numel() - batch + 1, batch):
            idx = order[k:k + batch]
            step_lr = lr * (0.5 * (1 + np.cos(np.pi * (ep + k / order.numel()) / epochs)))
            losses.append(net.train_step(dX[idx].contiguous(), dY[idx].contiguous(), step_lr))
        yv = torch.empty((vi.numel(), N_OUT), dtype=torch.float32, device="cuda")
        net.forward(dX[vi].contiguous(), yv)
        r2 = 1.0 - ((yv - dY[vi]) ** 2).mean(0).cpu().numpy()  # standardised targets: variance ~1
        hist.append((float(np.mean(losses)), [float(v) for v in r2]))
        log(f"epoch {ep}: train {np.mean(losses):.5f}, validation R^2 per output {np.round(r2, 4).tolist()}")
    torch.cuda.synchronize()
    return Surrogate(net, x_mu, x_sd, y_mu, y_sd), hist, time.time() - t0


def assimilate(sur, n_tr, members_per_group=128, spinup_tr=5, log=_log):
    """Surrogate-driven EnKF for G x members_per_group members with a simulated audit subset."""
    import torch

    ens = Ensemble("c4_ensemble", log=log)
    tb, lay = ens.tb, ens.lay
    cfg = ens.cfg
    G, Ma = lay.groups, lay.members
    Ms = members_per_group
    pr = cfg["prior"]
    rng = np.random.Generator(np.random.Philox(99))
    C = len(ens.cols)
    theta = (pr["log_gain_mean"] + pr["log_gain_sd"] * rng.standard_normal((C, Ms))).astype(np.float32)
    # the simulated audit members are the first Ma surrogate members (same draws)
    ens.theta = theta[:, :Ma].copy()
    ens.apply()
    model_var = None  # running mean square of the surrogate's BOLD error on the audit members
    col_vox = ens.vox_idx[:, Ma]  # the targets' voxels give each column's size and couplings
    sizes = np.diff(tb.voxel_start).astype(np.float64)
    logn = np.log(sizes[col_vox]) - 9.0
    # inter-voxel coupling between columns of the same group (targets' coupling rows)
    rows, cols_, vals = dti_matrix(tb, lay)
    colmap = -np.ones(tb.nv, np.int64)
    colmap[col_vox] = np.arange(C)
    keep = colmap[rows] >= 0
    P = (colmap[rows[keep]], colmap[cols_[keep]], vals[keep])
    # surrogate member states (per column, per member): previous rate, Balloon state, previous gain
    r_prev = np.full((C, Ms), 10.0)
    st_prev = np.zeros((4, C, Ms))
    st_prev[1:] = 1.0
    th_prev = theta.copy()
    dt_s = float(cfg["dt"]) * 1e-3
    obs_sd_rel = float(cfg["enkf"]["obs_sd_rel"])
    infl = float(cfg["enkf"]["inflation"])
    hist = []
    t_sim = t_sur = 0.0
    fallbacks = 0
    sim_theta = ens.theta  # the simulated audit members' parameters [C][Ma]
    for tr in range(spinup_tr + n_tr):
        # simulator: targets + audit members
        t0 = time.time()
        c0 = ens.net.voxel_spikes()
        ens.net.step(ens.tr_steps)
        rates_sim = (ens.net.voxel_spikes() - c0) / (sizes * ens.tr_steps * dt_s)
        y_all = ens.net.get_bold_samples()[-1].astype(np.float64)
        y_obs = y_all[col_vox]
        t1 = time.time()
        # surrogate: all members, one batched forward
        aff = np.zeros((C, Ms))
        for m in range(Ms):
            aff[:, m] = afferent(r_prev[:, m], P)
        th4 = np.stack([theta, theta, np.zeros_like(theta), np.zeros_like(theta)], -1)  # [C][Ms][4]
        feats = np.concatenate([th4, (r_prev / R_SCALE)[..., None], (st_prev[0] * S_SCALE)[..., None],
                                ((st_prev[1] - 1) * S_SCALE)[..., None], ((st_prev[2] - 1) * S_SCALE)[..., None],
                                ((st_prev[3] - 1) * S_SCALE)[..., None], (aff / R_SCALE)[..., None],
                                th_prev[..., None], np.broadcast_to(logn[:, None, None], (C, Ms, 1))], -1)
        x_dev = torch.from_numpy(feats.reshape(C * Ms, N_IN).astype(np.float32)).cuda()
        out = sur.predict(x_dev).cpu().numpy().reshape(C, Ms, N_OUT).astype(np.float64)
        r_new = np.maximum(out[..., 0] * R_SCALE, 0.0)
        y_sur = out[..., 1] / S_SCALE
        st_new = np.stack([out[..., 2] / S_SCALE, 1 + out[..., 3] / S_SCALE, 1 + out[..., 4] / S_SCALE,
                           1 + out[..., 5] / S_SCALE])
        t2 = time.time()
        # audit: the surrogate's rate for the simulated members, from their own simulated history
        audit_err = float("nan")
        if tr > 0:
            sv = ens.vox_idx[:, :Ma]
            a_th4 = np.stack([sim_theta, sim_theta, np.zeros_like(sim_theta), np.zeros_like(sim_theta)], -1)
            a_aff = np.stack([afferent(prev_sim_rates[sv[:, m]], P) for m in range(Ma)], 1)
            a_feat = np.concatenate([a_th4, (prev_sim_rates[sv] / R_SCALE)[..., None],
                                     (prev_sim_state[0][sv] * S_SCALE)[..., None],
                                     ((prev_sim_state[1][sv] - 1) * S_SCALE)[..., None],
                                     ((prev_sim_state[2][sv] - 1) * S_SCALE)[..., None],
                                     ((prev_sim_state[3][sv] - 1) * S_SCALE)[..., None], (a_aff / R_SCALE)[..., None],
                                     prev_sim_theta[..., None], np.broadcast_to(logn[:, None, None], (C, Ma, 1))], -1)
            xa = torch.from_numpy(a_feat.reshape(C * Ma, N_IN).astype(np.float32)).cuda()
            ya = sur.predict(xa)
            r_pred = np.maximum(ya.cpu().numpy()[:, 0].reshape(C, Ma) * R_SCALE, 0.0)
            r_true = rates_sim[sv]
            e2 = np.mean((ya.cpu().numpy()[:, 1].reshape(C, Ma) / S_SCALE - y_all[sv]) ** 2, 1)
            model_var = e2 if model_var is None else 0.7 * model_var + 0.3 * e2
            act = r_true >= 1.0
            audit_err = float(np.mean(np.abs(r_pred[act] - r_true[act]) / r_true[act]))
        _, sim_state = ens.net.get_bold()
        prev_sim_rates, prev_sim_state = rates_sim, sim_state.astype(np.float64)
        prev_sim_theta = sim_theta.copy()
        err = float(np.sqrt(np.mean((theta.mean(1) - ens.theta_star) ** 2)))
        corr = float(np.corrcoef(y_sur.mean(1), y_obs)[0, 1])
        used = "surrogate"
        t3 = time.time()
        if tr >= spinup_tr:
            sd = obs_sd_rel * np.maximum(np.abs(y_obs), 1e-4)
            fallback = not (audit_err <= 0.05)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
            if fallback:
                # the plain simulator decides this TR: analysis of the simulated audit members, and the
                # surrogate ensemble is re-centred on their analysed mean (its spread kept)
                fallbacks += 1
                used = "simulator"
                hx = y_all[ens.vox_idx[:, :Ma]]
                th = t(theta[:, :Ma])
                dtb.dtb_enkf_analysis(th, t(hx), t(y_obs), t(sd), t(rng.standard_normal(hx.shape)), inflation=infl)
                theta += (th.cpu().numpy().mean(1) - theta.mean(1))[:, None]
            else:
                # observation error = measurement noise + the surrogate's own error (audit members)
                sd_m = np.sqrt(sd * sd + (model_var if model_var is not None else 0.0))
                th = t(theta)
                dtb.dtb_enkf_analysis(th, t(y_sur), t(y_obs), t(sd_m), t(rng.standard_normal(y_sur.shape)),
                                   inflation=infl)
                theta = th.cpu().numpy()
            # the simulated audit members follow the surrogate ensemble's analysis (first Ma members)
            ens.theta = theta[:, :Ma].copy()
            ens.apply()
            sim_theta = ens.theta
        th_prev = theta.copy()
        r_prev, st_prev = r_new, st_new
        t4 = time.time()
        t_sim += t1 - t0
        t_sur += (t2 - t1) + (t4 - t3)
        hist.append({"tr": tr, "param_rmse": err, "bold_corr": corr, "audit_rate_err": audit_err, "used": used})
        if tr % 5 == 0 or tr == spinup_tr + n_tr - 1:
            log(f"TR {tr}: RMSE {err:.4f}, BOLD corr {corr:.3f}, audit rate error {audit_err:.3f}, {used}")
    ens.close()
    return hist, t_sim, t_sur, fallbacks, C


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--windows", type=int, default=150)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--n-tr", type=int, default=40)
    ap.add_argument("--members", type=int, default=128)
    ap.add_argument("--save-model", default=None, help="write the trained surrogate (.npz)")
    ap.add_argument("--load-model", default=None, help="skip data and training, use this surrogate (.npz)")
    a = ap.parse_args()
    if a.load_model:
        sur, hist_train, train_s, gen_s, n_rows = Surrogate.load(a.load_model), [(float("nan"), [])], 0.0, 0.0, 0
    else:
        X, Y, gen_s = generate(a.windows)
        n_rows = int(X.shape[0])
        _log(f"dataset: {n_rows} windows in {gen_s:.1f} s")
        sur, hist_train, train_s = train(X, Y, epochs=a.epochs)
        if a.save_model:
            sur.save(a.save_model)
    hist, t_sim, t_sur, fallbacks, C = assimilate(sur, a.n_tr, members_per_group=a.members)
    sur.close()
    ens_steps = 72  # networks the simulator runs per step in the audit setup (8 targets + 64 audit members)
    sim_cost_per_tr = t_sim / len(hist)
    full_sim_cost = sim_cost_per_tr * (8 * (a.members + 1)) / ens_steps
    res = {
        "dataset_windows": n_rows, "generate_s": gen_s, "train_s": train_s, "model_loaded": a.load_model,
        "train_loss_by_epoch": [round(h[0], 6) for h in hist_train],
        "val_r2_by_output": [round(v, 4) for v in hist_train[-1][1]],
        "outputs": ["rate", "bold_y", "s", "f", "v", "q"],
        "members": 8 * a.members, "columns": C, "n_tr": a.n_tr,
        "prior_rmse": hist[0]["param_rmse"], "final_rmse": hist[-1]["param_rmse"],
        "final_bold_corr": hist[-1]["bold_corr"],
        "rmse_by_tr": [round(h["param_rmse"], 5) for h in hist],
        "audit_rate_err_by_tr": [None if not np.isfinite(h["audit_rate_err"]) else round(h["audit_rate_err"], 4)
                                 for h in hist],
        "fallback_trs": fallbacks,
        "sim_s_per_tr_audit": sim_cost_per_tr, "surrogate_s_per_tr": t_sur / len(hist),
        "sim_s_per_tr_for_all_members_estimated": full_sim_cost,
        "speedup_vs_simulating_all_members": full_sim_cost / (sim_cost_per_tr + t_sur / len(hist)),
    }
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
