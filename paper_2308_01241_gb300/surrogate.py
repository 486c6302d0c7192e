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

Phases (``run``; the GPU test ``tests/test_gpu_surrogate.py`` runs a small
case of the same code):

1. **Data.** The simulator runs a merged ensemble network (groups of
   uneven size, every copy of a group one network). The hyper-parameters of
   every voxel follow an AR(1) walk across windows around the prior
   (correlation 0.8 per window), so the previous window's state is
   informative as it is during assimilation, where the EnKF moves the
   parameters a little per TR. Every window gives one (input, output) row
   per voxel.
2. **Training.** Inputs and targets are standardised with the training rows'
   mean and standard deviation; Adam on mini-batches, on the GPU.
3. **Simulator-driven assimilation** (the method without the surrogate):
   M members per column and one hidden target per group, all simulated, the
   cycle run by ``dtb_assimilate``. Its targets' BOLD is the observation
   sequence of both arms.
4. **Surrogate-driven assimilation**, the same M members, prior draws and
   observations. The simulator runs only an audit subset of A members per
   column (members 0 .. A-1: about 5 %); the surrogate predicts all M.
   Every TR:
   - the audit members anchor the ensemble: their simulated window replaces
     their prediction, and the column's mean prediction error on them (all
     six outputs) is subtracted from every other member, so that the
     rolled-forward surrogate states do not drift; the spread of the
     remaining BOLD error is added to the observation noise;
   - the surrogate alone is checked on the audit members (from their own
     simulated previous window): the rate-weighted error of the columns'
     mean audit rate, and the error of the rate spread across the audit
     members relative to the mean rate;
   - if either exceeds 5 %, the TR falls back to the plain simulator: no
     surrogate analysis is made, and the simulated audit members keep the
     ensemble anchored until the surrogate agrees with them again
     (``on_fallback="recentre"`` instead re-centres the ensemble on an
     analysis of the audit members alone);
   - otherwise the EnKF analysis uses the surrogate's predictions of all M.
   Both arms are timed per TR on the same GPU, and their recovered
   parameters (RMSE against the hidden targets) and BOLD fit (Pearson of
   the ensemble-mean prediction with the observation) are compared.

    python -m paper_2308_01241_gb300.surrogate [--groups 2 --members 128 --audit 6]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import dtb, netgen
from .surrogate_mlp import MLP

N_IN, WIDTH, DEPTH, N_OUT = 12, 256, 3, 6
R_SCALE = 20.0    # Hz
S_SCALE = 100.0   # Balloon states and BOLD around rest


def _log(*m):
    print(*m, file=sys.stderr, flush=True)


def dti_matrix(tb):
    """Row-normalised inter-voxel coupling P[v, u] of the merged network, as (rows, cols, values)."""
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


def ensemble_network(cfg, groups, copies, vox_range, neuron_range, delivery="bins"):
    """A merged ensemble network of `groups` groups with `copies` networks each
    (netgen's last copy of a group is called its target there): (net, tb, lay, csr)."""
    tb, lay = netgen.make_ensemble_tables(cfg, groups, copies - 1, vox_range, neuron_range)
    csr = netgen.device_csr(tb, cfg["wfmt"])
    tr = int(cfg["enkf"]["tr_steps"])
    net = dtb.Network(n=tb.n, voxel_start=tb.voxel_start, vparams=tb.vparams(1.0), delay_vv=tb.delay_vv,
                      d_max=tb.d_max, csr=csr, wfmt=cfg["wfmt"], wshift=4, n_ch=int(cfg["n_ch"]),
                      dt=float(cfg["dt"]), nu_ext=float(cfg["nu_ext"]), w_ext=int(cfg["w_ext"]),
                      seed=int(cfg["seeds"]["drive"]), init_seed=int(cfg["seeds"]["init"]), bold=cfg["bold"],
                      bold_every=tr, delivery=delivery, log_capacity=1 << 16)
    return net, tb, lay, csr


def column_voxels(lay):
    """[C][copies] voxel (in the merged network) of every column (a voxel of a
    group) in every copy of its group."""
    cols = []
    for g, V in enumerate(lay.group_vox):
        for v in range(V):
            cols.append([o + v for o, _ in lay.net_vox[g]])
    return np.array(cols, np.int64)


def generate(net, tb, n_windows, tr_steps, seed=2024, log=_log):
    """Simulator windows of a network with AR(1) hyper-parameters per voxel: (X, Y, seconds)."""
    rng = np.random.default_rng(seed)
    base = tb.vparams(1.0)
    sizes = np.diff(tb.voxel_start).astype(np.float64)
    logn = np.log(sizes) - 9.0
    P = dti_matrix(tb)
    dt_s = float(tb.cfg["dt"]) * 1e-3
    X, Y = [], []
    prev = None
    t0 = time.time()
    rho = 0.8
    mean4 = np.array([0.18, 0.18, 0.0, 0.0])
    sd4 = np.array([0.12, 0.12, 0.05, 0.05])
    th4 = mean4 + sd4 * rng.standard_normal((tb.nv, 4))
    net.reset()
    for w in range(n_windows + 1):
        th4 = mean4 + rho * (th4 - mean4) + np.sqrt(1 - rho * rho) * sd4 * rng.standard_normal((tb.nv, 4))
        th4[:, 1] = th4[:, 0] + 0.02 * rng.standard_normal(tb.nv)
        thA = th4[:, 0].copy()
        net.set_hyperparams(base[:, 6:10] * np.exp(th4))
        c0 = net.voxel_spikes()
        net.step(tr_steps)
        rate = (net.voxel_spikes() - c0) / (sizes * tr_steps * dt_s)
        y, st = net.get_bold()
        st = st.astype(np.float64)
        if prev is not None:
            r_prev, st_prev, thA_prev = prev
            X.append(features(th4, r_prev, st_prev, afferent(r_prev, P), thA_prev, logn))
            Y.append(targets(rate, y.astype(np.float64), st))
        prev = (rate, st, thA)
        if w % 10 == 0:
            log(f"window {w}: {time.time() - t0:.1f} s, mean rate {rate.mean():.2f} Hz")
    net.reset()
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


def _rmse(theta, theta_star):
    return float(np.sqrt(np.mean((theta.mean(1) - theta_star) ** 2)))


def _corr(pred, obs):
    return float(np.corrcoef(pred, obs)[0, 1]) if np.std(pred) > 0 and np.std(obs) > 0 else float("nan")


def simulator_driven(net, tb, lay, theta0, theta_star, n_tr, spinup_tr=4, obs_sd_rel=0.02, inflation=1.03,
                     seed=16, log=_log):
    """The method without the surrogate: every member simulated, the cycle run by
    dtb_assimilate (predict, gather, EnKF, re-sampling on the GPU).  Members are
    copies 0 .. M-1 of every group, the hidden target its last copy."""
    cfg = tb.cfg
    tr = int(cfg["enkf"]["tr_steps"])
    cv = column_voxels(lay)
    M = theta0.shape[1]
    base = tb.vparams(1.0)
    g = base[:, 6:10].copy()
    g[cv[:, -1], 0] *= np.exp(theta_star)
    g[cv[:, -1], 1] *= np.exp(theta_star)
    net.reset()
    net.set_hyperparams(g)
    asm = dtb.Assimilation(net, cv[:, :M], theta0, base[:, 6:10], tr, target_voxel=cv[:, -1], obs_sd_rel=obs_sd_rel,
                           inflation=inflation, seed=seed)
    t0 = time.time()
    net.step(spinup_tr * tr)
    t1 = time.time()
    th, hx, y = asm.assimilate(n_tr)
    t2 = time.time()
    asm.close()
    hist = [{"tr": -1, "param_rmse": _rmse(theta0, theta_star), "bold_corr": float("nan")}]
    for k in range(n_tr):
        hist.append({"tr": k, "param_rmse": _rmse(th[k], theta_star), "bold_corr": _corr(hx[k].mean(1), y[k])})
    log(f"simulator-driven: {M} members, RMSE {hist[0]['param_rmse']:.4f} -> {hist[-1]['param_rmse']:.4f}, "
        f"BOLD r {hist[-1]['bold_corr']:.3f}, {(t2 - t1) / n_tr:.3f} s per TR")
    return {"history": hist, "y_obs": y.astype(np.float64), "s_per_tr": (t2 - t1) / n_tr,
            "spinup_s_per_tr": (t1 - t0) / max(spinup_tr, 1), "theta": th[-1]}


def surrogate_driven(sur, net, tb, lay, theta0, theta_star, y_obs, spinup_tr=4, obs_sd_rel=0.02, inflation=1.03,
                     err_limit=0.05, seed=99, audit_metric="pooled", on_fallback="skip", log=_log):
    """The surrogate in the predict step for all M members; the simulator runs
    only the audit members, members 0 .. A-1 of every column (the copies of the
    audit network's groups, given those members' parameters), and is the
    fallback.  y_obs [n_tr][C]: the observations of the analysis TRs (after
    spinup_tr spin-up TRs).

    Every TR the audit members anchor the ensemble: their simulated window
    replaces their surrogate prediction, and the column's mean prediction
    error on them (all six outputs, rate and BOLD and Balloon states) is
    subtracted from every other member's prediction, so that the rolled-forward
    surrogate states do not drift from the simulated ones.  The spread of the
    remaining BOLD error is added to the observation noise."""
    import torch

    cfg = tb.cfg
    tr_steps = int(cfg["enkf"]["tr_steps"])
    rng = np.random.default_rng(seed)
    cv = column_voxels(lay)
    C, A = cv.shape
    M = theta0.shape[1]
    n_tr = y_obs.shape[0]
    theta = theta0.astype(np.float64).copy()
    sizes = np.diff(tb.voxel_start).astype(np.float64)
    logn = np.log(sizes[cv[:, 0]]) - 9.0
    rows, cols_, vals = dti_matrix(tb)
    colmap = -np.ones(tb.nv, np.int64)
    colmap[cv[:, 0]] = np.arange(C)
    keep = colmap[rows] >= 0
    Pd = np.zeros((C, C))  # coupling between the columns (each group's voxels), dense
    np.add.at(Pd, (colmap[rows[keep]], colmap[cols_[keep]]), vals[keep])
    base = tb.vparams(1.0)
    dt_s = float(cfg["dt"]) * 1e-3

    def apply_audit():
        g = base[:, 6:10].copy()
        gain = np.exp(theta[:, :A])
        g[cv.ravel(), 0] *= gain.ravel()
        g[cv.ravel(), 1] *= gain.ravel()
        net.set_hyperparams(g)

    def predict(th, r_prev, st_prev, th_prev, m):
        """Surrogate outputs [C][m][6] (rate / R_SCALE, y and Balloon states scaled) of m members."""
        aff = Pd @ r_prev  # the DTI-weighted rate of each member's source voxels
        z = np.zeros_like(th)
        f = np.concatenate([np.stack([th, th, z, z], -1), (r_prev / R_SCALE)[..., None],
                            (st_prev[0] * S_SCALE)[..., None], ((st_prev[1] - 1) * S_SCALE)[..., None],
                            ((st_prev[2] - 1) * S_SCALE)[..., None], ((st_prev[3] - 1) * S_SCALE)[..., None],
                            (aff / R_SCALE)[..., None], th_prev[..., None],
                            np.broadcast_to(logn[:, None, None], (C, m, 1))], -1)
        x = torch.from_numpy(f.reshape(C * m, N_IN).astype(np.float32)).cuda()
        return sur.predict(x).cpu().numpy().reshape(C, m, N_OUT).astype(np.float64)

    def unpack(out):
        r = np.maximum(out[..., 0] * R_SCALE, 0.0)
        st = np.stack([out[..., 2] / S_SCALE, 1 + out[..., 3] / S_SCALE, 1 + out[..., 4] / S_SCALE,
                       1 + out[..., 5] / S_SCALE])
        return r, out[..., 1] / S_SCALE, st

    net.reset()
    apply_audit()
    r_prev = np.full((C, M), 10.0)
    st_prev = np.zeros((4, C, M))
    st_prev[1:] = 1.0
    th_prev = theta.copy()
    sim_prev = None  # the audit members' simulated previous window: rate [C][A], Balloon state [4][C][A], gains
    resid = None
    hist = [{"tr": -1, "param_rmse": _rmse(theta, theta_star), "bold_corr": float("nan")}]
    t_sim = t_sur = 0.0
    tr_times = []  # (simulation, surrogate) seconds of every TR
    fallbacks = 0
    for tr in range(spinup_tr + n_tr):
        t0 = time.time()
        c0 = net.voxel_spikes()
        net.step(tr_steps)
        rates_all = (net.voxel_spikes() - c0) / (sizes * tr_steps * dt_s)
        y_all = net.get_bold_samples()[-1].astype(np.float64)
        _, st_all = net.get_bold()
        torch.cuda.synchronize()  # every stream of the simulation is done: its time ends here
        t1 = time.time()
        r_sim, y_sim = rates_all[cv], y_all[cv]
        st_sim = st_all.astype(np.float64)[:, cv]
        sim_out = targets(r_sim.ravel(), y_sim.ravel(), st_sim.reshape(4, -1)).astype(np.float64).reshape(C, A, N_OUT)
        out = predict(theta, r_prev, st_prev, th_prev, M)
        drift = (out[:, :A] - sim_out).mean(1)  # the column's prediction error on its audit members
        err_y = (out[:, :A, 1] - sim_out[..., 1] - drift[:, None, 1]) / S_SCALE
        v = (err_y ** 2).mean(1)
        resid = v if resid is None else 0.7 * resid + 0.3 * v
        out = out - drift[:, None, :]
        out[:, :A] = sim_out  # the audit members are simulated exactly
        r_new, y_sur, st_new = unpack(out)
        audit_err = spread_err = float("nan")
        if sim_prev is not None:
            # the surrogate alone on the audit members (from their simulated previous window): the mean
            # rate of each column's audit members, and the rate spread across them
            pr, pst, pth = sim_prev
            r_pred = np.maximum(predict(theta[:, :A], pr, pst, pth, A)[..., 0] * R_SCALE, 0.0)
            ok = r_sim.mean(1) >= 1.0
            if audit_metric == "pooled":  # rate-weighted over the subset: sum |error| / sum rate
                audit_err = float(np.abs(r_pred[ok].mean(1) - r_sim[ok].mean(1)).sum() / r_sim[ok].mean(1).sum())
            else:  # per column, then averaged
                audit_err = float(np.mean(np.abs(r_pred[ok].mean(1) - r_sim[ok].mean(1)) / r_sim[ok].mean(1)))
            spread_err = float(abs(np.sqrt(r_pred[ok].var(1).mean()) - np.sqrt(r_sim[ok].var(1).mean()))
                               / r_sim[ok].mean())
        sim_prev = (r_sim, st_sim, theta[:, :A].copy())
        if tr >= spinup_tr:
            k = tr - spinup_tr
            y = y_obs[k]
            sd = obs_sd_rel * np.maximum(np.abs(y), 1e-4)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
            corr = _corr(y_sur.mean(1), y)
            if not (audit_err <= err_limit and spread_err <= err_limit):
                fallbacks += 1
                used = "simulator"
                if on_fallback == "recentre":
                    # the plain simulator decides: analysis of the simulated audit members, and the
                    # surrogate ensemble re-centred on their analysed mean (its spread kept)
                    th = t(theta[:, :A])
                    dtb.dtb_enkf_analysis(th, t(y_sim), t(y), t(sd), t(rng.standard_normal((C, A))),
                                          inflation=inflation)
                    theta += (th.cpu().numpy().astype(np.float64).mean(1) - theta.mean(1))[:, None]
                # on_fallback == "skip": no analysis this TR; the simulated audit members keep the
                # ensemble anchored until the surrogate agrees with them again
            else:
                used = "surrogate"
                sd_m = np.sqrt(sd * sd + resid)
                th = t(theta)
                dtb.dtb_enkf_analysis(th, t(y_sur), t(y), t(sd_m), t(rng.standard_normal((C, M))), inflation=inflation)
                theta = th.cpu().numpy().astype(np.float64)
            apply_audit()
            hist.append({"tr": k, "param_rmse": _rmse(theta, theta_star), "bold_corr": corr, "used": used,
                         "audit_rate_err": audit_err, "spread_err": spread_err})
        th_prev = theta.copy()
        r_prev, st_prev = r_new, st_new
        torch.cuda.synchronize()
        t2 = time.time()
        if tr >= spinup_tr:  # the analysis TRs, as the simulator-driven arm's time per TR
            t_sim += t1 - t0
            t_sur += t2 - t1
        tr_times.append((t1 - t0, t2 - t1))
    n_all = n_tr
    log(f"surrogate-driven: {M} members ({A} audit), RMSE {hist[0]['param_rmse']:.4f} -> "
        f"{hist[-1]['param_rmse']:.4f}, BOLD r {hist[-1]['bold_corr']:.3f}, {fallbacks} fallbacks, "
        f"{(t_sim + t_sur) / n_all:.3f} s per TR (simulator {t_sim / n_all:.3f}, surrogate {t_sur / n_all:.4f})")
    return {"history": hist, "s_per_tr": (t_sim + t_sur) / n_all, "sim_s_per_tr": t_sim / n_all,
            "surrogate_s_per_tr": t_sur / n_all, "fallbacks": fallbacks, "theta": theta, "tr_times": tr_times}


def run(groups=2, members=128, audit=6, vox_range=(20, 30), neuron_range=(50000, 70000), windows=30, epochs=8,
        n_tr=12, spinup_tr=4, autotune=True, log=_log):
    """Data, training and both assimilation arms on one GPU; returns the report.
    With autotune, each arm's network runs with the launch shapes dtb_autotune
    picks for it (the small audit network and the full ensemble differ)."""
    import torch

    cfg = netgen.load_config("c4_ensemble")
    tr_steps = int(cfg["enkf"]["tr_steps"])
    vr, nr = list(vox_range), list(neuron_range)
    t0 = time.time()
    net, tb, lay, csr = ensemble_network(cfg, groups, members + 1, vr, nr)
    log(f"simulated ensemble: {tb.n} neurons, {tb.nv} voxels, {tb.n * tb.K:.3g} synapses, setup "
        f"{time.time() - t0:.1f} s")
    shapes = {}
    if autotune:
        shapes["simulator_driven"] = net.autotune(20)
        net.reset()
        log(f"launch shapes of the full ensemble: {shapes['simulator_driven']}")
    X, Y, gen_s = generate(net, tb, windows, tr_steps, log=log)
    sur, hist_train, train_s = train(X, Y, epochs=epochs, log=log, max_batch=1 << 18)
    C = len(column_voxels(lay))
    pr = cfg["prior"]
    rng = np.random.Generator(np.random.Philox(int(cfg["seeds"]["prior"])))
    theta0 = (pr["log_gain_mean"] + pr["log_gain_sd"] * rng.standard_normal((C, members))).astype(np.float32)
    theta_star = pr["log_gain_mean"] + pr["log_gain_sd"] * rng.standard_normal(C)
    sim = simulator_driven(net, tb, lay, theta0, theta_star, n_tr, spinup_tr=spinup_tr,
                           obs_sd_rel=float(cfg["enkf"]["obs_sd_rel"]), inflation=float(cfg["enkf"]["inflation"]),
                           seed=int(cfg["seeds"]["enkf"]), log=log)
    net.close()
    del csr
    torch.cuda.empty_cache()
    net_a, tb_a, lay_a, csr_a = ensemble_network(cfg, groups, audit, vr, nr)
    assert lay_a.group_vox == lay.group_vox
    if autotune:
        shapes["surrogate_driven"] = net_a.autotune(20)
        net_a.reset()
        log(f"launch shapes of the audit network: {shapes['surrogate_driven']}")
    srg = surrogate_driven(sur, net_a, tb_a, lay_a, theta0, theta_star, sim["y_obs"], spinup_tr=spinup_tr,
                           obs_sd_rel=float(cfg["enkf"]["obs_sd_rel"]), inflation=float(cfg["enkf"]["inflation"]),
                           log=log)
    net_a.close()
    sur.close()
    return {
        "groups": groups, "columns": C, "members": members, "audit_members": audit, "group_voxels": lay.group_vox,
        "simulated_neurons": {"simulator_driven": int(tb.n), "surrogate_driven": int(tb_a.n)},
        "dataset_rows": int(X.shape[0]), "generate_s": gen_s, "train_s": train_s,
        "val_r2_by_output": [round(v, 4) for v in hist_train[-1][1]],
        "outputs": ["rate", "bold_y", "s", "f", "v", "q"], "n_tr": n_tr, "spinup_tr": spinup_tr,
        "prior_rmse": sim["history"][0]["param_rmse"],
        "simulator_driven": {"final_rmse": sim["history"][-1]["param_rmse"],
                             "final_bold_corr": sim["history"][-1]["bold_corr"], "s_per_tr": sim["s_per_tr"],
                             "rmse_by_tr": [round(h["param_rmse"], 5) for h in sim["history"]]},
        "surrogate_driven": {"final_rmse": srg["history"][-1]["param_rmse"],
                             "final_bold_corr": srg["history"][-1]["bold_corr"], "s_per_tr": srg["s_per_tr"],
                             "sim_s_per_tr": srg["sim_s_per_tr"], "surrogate_s_per_tr": srg["surrogate_s_per_tr"],
                             "fallback_trs": srg["fallbacks"],
                             "rmse_by_tr": [round(h["param_rmse"], 5) for h in srg["history"]],
                             "used_by_tr": [h.get("used") for h in srg["history"][1:]],
                             "audit_rate_err_by_tr": [round(h["audit_rate_err"], 4) for h in srg["history"][1:]],
                             "spread_err_by_tr": [round(h["spread_err"], 4) for h in srg["history"][1:]],
                             "sim_and_surrogate_s_by_tr": [[round(a, 4), round(b, 4)] for a, b in srg["tr_times"]]},
        "speedup": sim["s_per_tr"] / srg["s_per_tr"],
        "launch_shapes": shapes,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--groups", type=int, default=2)
    ap.add_argument("--members", type=int, default=128)
    ap.add_argument("--audit", type=int, default=6)
    ap.add_argument("--vox-range", type=int, nargs=2, default=[20, 30])
    ap.add_argument("--neuron-range", type=int, nargs=2, default=[50000, 70000])
    ap.add_argument("--windows", type=int, default=30)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--n-tr", type=int, default=12)
    ap.add_argument("--spinup-tr", type=int, default=4)
    ap.add_argument("--no-autotune", action="store_true", help="library default launch shapes for both networks")
    a = ap.parse_args()
    res = run(a.groups, a.members, a.audit, a.vox_range, a.neuron_range, a.windows, a.epochs, a.n_tr, a.spinup_tr,
              autotune=not a.no_autotune)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
