"""Learned column closure: training data from fine LES, training, coarse runs, errors.

The workflow the paper motivates for calibrated closures (Sec. 3.2.3: a parameterisation tuned
against a suite of LES) done with this library's own kernels:

1. A batched ensemble of fine convective boundary-layer LES (uneven sizes and forcings) is
   stepped on the GPU.  At regular times every member is box-filtered onto a coarse horizontal
   grid (``Model.coarse_grain``): the coarse state and the subfilter vertical fluxes tau of b,
   ubar and vbar that a coarse model cannot resolve.
2. The coarse state is loaded into a coarse model of the same forcing; its raw column features
   (``Model.closure_features``) are the network inputs and tau minus the coarse model's own AMD
   vertical flux (``Model.column_fluxes``) at the interior faces is the target: the network
   learns what AMD misses.
3. The network (``ocn.MLP``, BF16 tensor-core GEMMs, hand-written backward pass and Adam) is
   trained on the training members' samples.
4. Coarse models of every forcing are run from the coarse-grained initial state with plain AMD
   and with AMD + the learned closure; their horizontal-mean b and total buoyancy-flux profiles
   are compared with those of the fine LES at the same times.

Everything runs through the CUDA library; numpy only sizes and summarises.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, ocn

FEATURES_USED = 20


def coarse_config(p: dict, cx: int = 16, cy: int = 16) -> dict:
    """The coarse-grid version of a workload dict: the same domain, vertical grid and forcing."""
    q = dict(p)
    q.update(Nx=cx, Ny=cy, name=p.get("name", "member") + f"_coarse{cx}x{cy}")
    return q


def _time_steps(t_end: float, dt: float) -> int:
    return int(round(t_end / dt))


def fine_run(members, t_end: float, dt: float, every: int, cx: int = 16, cy: int = 16, on_snapshot=None,
             seed: int = inputs.SEED):
    """Step the fine ensemble to t_end, calling on_snapshot(step, ensemble) every `every` steps
    (and at step 0).  Returns the per-member profile series [(t, profiles dict)]."""
    ens = ocn.Ensemble(members)
    for i, (p, m) in enumerate(zip(members, ens.members)):
        m.set(**inputs.initial_state(p, seed=seed + p.get("member", i)))
    ens.autotune()
    n = _time_steps(t_end, dt)
    series = [[] for _ in members]
    for step in range(0, n + 1, every):
        if step > 0:
            ens.time_step(dt, every)
        ens.synchronize()
        for i, m in enumerate(ens.members):
            series[i].append((step * dt, m.profiles()))
        if on_snapshot is not None:
            on_snapshot(step, ens)
    return ens, series


def training_samples(members, coarse_models, ens, cx: int, cy: int, target: str = "column"):
    """(X, Y, G) device tensors of one snapshot: raw features, targets tau - F_closure and the
    member index, at the interior faces of every coarse column of every member.  target
    "column" keeps each column's own subfilter flux; "mean" replaces it by the member's
    horizontal mean at that face (the part the mean profiles feel, without subgrid noise)."""
    import torch
    Xs, Ys, Gs = [], [], []
    for idx, (p, fine, coarse) in enumerate(zip(members, ens.members, coarse_models)):
        c = fine.coarse_grain(cx, cy)
        coarse.set(project=False, u=c["u"], v=c["v"], w=c["w"], b=c["b"])
        X = coarse.closure_features(p["N2"])
        F = coarse.column_fluxes().double()
        Nz = p["Nz"]
        res = c["tau"] - F                                         # [3][Nz+1][cy][cx]
        if target == "mean":
            res = res.mean(dim=(2, 3), keepdim=True).expand_as(res)
        tgt = res.reshape(3, -1).t()                               # [(Nz+1)*cy*cx][3], sample order k, j, i
        k = torch.arange((Nz + 1) * cx * cy, device=X.device) // (cx * cy)
        keep = (k >= 1) & (k <= Nz - 1)
        Xs.append(X[keep])
        Ys.append(tgt[keep].float())
        Gs.append(torch.full((int(keep.sum()),), idx, dtype=torch.int32, device=X.device))
    return torch.cat(Xs), torch.cat(Ys), torch.cat(Gs)


def normalisation(X):
    """Per-feature mean and scale over the samples (constant features scaled by their magnitude)."""
    Xn = X[:, :FEATURES_USED].double()
    mu = np.zeros(ocn.COLUMN_FEATURES)
    sigma = np.ones(ocn.COLUMN_FEATURES)
    m = Xn.mean(dim=0).cpu().numpy()
    sd = Xn.std(dim=0).cpu().numpy()
    const = sd <= 1e-6 * np.abs(m)
    mu[:FEATURES_USED] = m
    sigma[:FEATURES_USED] = np.where(const, np.maximum(np.abs(m), 1e-30), np.where(sd > 0, sd, 1.0))
    # the mixed-layer depth is a length like the face depth: never scale it below a thousandth of the
    # depths' spread, so that a column without a mixed layer (h at rounding level) stays near zero
    sigma[19] = max(sigma[19], 1e-3 * sigma[18])
    return mu, sigma


NONLOCAL = (15, 16, 17, 18, 19)      # Jb, f, N2, depth, mixed-layer depth: no local gradients
LOCAL = tuple(range(17))             # db/dz, dubar/dz, dvbar/dz at the five faces k-2..k+2, Jb, f
# The trained closure: the buoyancy flux (momentum stays with AMD), non-dimensionalised by the
# surface buoyancy flux, from the non-local features only, fitted to the member-mean residual.
# Feeding the local gradients as well fits the training data better but feeds grid-scale
# gradients back into the explicit flux and degrades the coupled runs.
DEFAULT_VARIANT = dict(target="mean", outputs=(0,), features="nonlocal", scale="Jb")
# The closure on the inputs the configuration states (local gradients of b, ubar, vbar over five
# faces, the surface buoyancy flux and f) in diffusivity form: the network predicts eddy
# diffusivities kappa (tracers) and nu (momentum) >= 0 at every face, whose column means the
# coarse model applies through its semi-implicit vertical solve.  The targets are capped at
# KAPPA_MAX and every face counts alike (a scan of the cap on a 32-forcing, 3 h experiment:
# 1, 0.1, 0.01, 0.005, 0.003, 0.001 m^2/s; 0.003 gave the lowest buoyancy-profile error, larger
# caps over-mix the stratified interior; weighting the faces by the squared gradient, the
# least-squares weight of the flux, fitted the mixed layer worse).
DIFFUSIVITY_VARIANT = dict(target="mean", outputs=(0, 1), features="local", form="diffusivity",
                           weighting="uniform", kmax=0.003)
KAPPA_MAX = 0.003                    # m^2/s: cap of the diffusivity targets


def diffusivity_targets(X, Y, ncol: int, kmax: float = KAPPA_MAX):
    """Per-sample diffusivity targets and least-squares weights from the member-mean residual
    fluxes Y [N][3] (one value per face, repeated over the ncol columns of a snapshot) and the
    column-mean gradients at the face (features 2, 7, 12): the flux -K g with the smallest
    squared error is K = -F g / g^2, clipped to [0, kmax]; its weight is g^2 (so that sampling
    in proportion to it makes the mean-square error of K the flux error)."""
    import torch
    gm = X[:, [2, 7, 12]].double().reshape(-1, ncol, 3).mean(dim=1)          # per face and snapshot
    gm = gm.repeat_interleave(ncol, dim=0)
    Yd = Y.double()
    gb = gm[:, 0]
    gb2 = gb * gb
    kap = torch.where(gb2 > 0, -Yd[:, 0] * gb / gb2.clamp_min(1e-300), torch.zeros_like(gb)).clamp(0.0, kmax)
    gu2 = gm[:, 1] ** 2 + gm[:, 2] ** 2
    nu = torch.where(gu2 > 0, -(Yd[:, 1] * gm[:, 1] + Yd[:, 2] * gm[:, 2]) / gu2.clamp_min(1e-300),
                     torch.zeros_like(gb)).clamp(0.0, kmax)
    T = torch.stack([kap, nu, torch.zeros_like(kap)], dim=1).float()
    w = gb2 / gb2.mean().clamp_min(1e-300) + gu2 / gu2.mean().clamp_min(1e-300)
    return T, w


def train(X, Y, steps: int = 3000, batch: int = 16384, lr: float = 1e-3, seed: int = inputs.SEED, log_every=0,
          outputs=(0, 1, 2), features=None, yscale=None, weights=None):
    """Train a 32-128-128-128-16 network on (X raw features, Y targets [N][3]); only the flux
    components in `outputs` enter the loss (the others get out_scale 0: the closure leaves them
    to the model's own closure); `features` (indices) restricts the inputs (the others are
    normalised to zero by an infinite scale); yscale [N][3] divides the targets per sample
    (e.g. by the member's surface buoyancy flux); weights [N] (or None) sets the probability
    with which a sample enters a batch, so that the mean-square loss is weighted by it.  Returns
    the network, the feature normalisation, the output scales and the loss history."""
    import torch
    mu, sigma = normalisation(X)
    if features is not None:
        for q in range(FEATURES_USED):
            if q not in features:
                mu[q], sigma[q] = 0.0, 1e30
    dev = X.device
    if yscale is not None:
        Y = (Y.double() / yscale.double()).float()
    out_scale = Y.double().std(dim=0).clamp_min(1e-30).cpu().numpy()
    Xn = ((X.double() - torch.tensor(mu, device=dev)) / torch.tensor(sigma, device=dev)).float()
    Xn[:, FEATURES_USED:] = 0.0
    Yn = torch.zeros((Y.shape[0], 16), dtype=torch.float32, device=dev)
    Yn[:, :3] = (Y.double() / torch.tensor(out_scale, device=dev)).float()
    mask = torch.zeros(16, dtype=torch.float32, device=dev)
    for q in outputs:
        mask[q] = 1.0
    for q in range(3):
        if q not in outputs:
            out_scale[q] = 0.0
    net = ocn.MLP(inputs.MLP_SIZES, max_batch=batch)
    net.set_params(inputs.mlp_init(seed=seed))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hist = []
    for s in range(steps):
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))        # cosine decay
        if weights is None:
            idx = torch.randint(0, Xn.shape[0], (batch,), device=dev, generator=g)
        else:
            idx = torch.multinomial(weights, batch, replacement=True, generator=g)
        loss = net.train_step(Xn[idx], Yn[idx], mask, lr_s)
        hist.append(loss)
        if log_every and s % log_every == 0:
            print(f"  step {s} loss {loss:.4f}", flush=True)
    return net, mu, sigma, out_scale, hist


def predict(net, mu, sigma, out_scale, X, chunk: int = 0):
    """Fluxes [N][3] the trained network predicts for raw features X (device tensors)."""
    import torch
    dev = X.device
    out = []
    chunk = chunk or net.max_batch
    for s in range(0, X.shape[0], chunk):
        Xc = ((X[s:s + chunk].double() - torch.tensor(mu, device=dev)) / torch.tensor(sigma, device=dev)).float()
        Xc[:, FEATURES_USED:] = 0.0
        y = net.forward(Xc)[:, :3].double()
        out.append(y * torch.tensor(out_scale, device=dev))
    return torch.cat(out)


def coarse_run(members, init_states, t_end: float, dt: float, every: int, closure=None):
    """Coarse ensemble from the given initial states; closure = (net, mu, sigma, out_scale[, mode])
    or a function p -> that tuple (per-member scales), or None (plain AMD); mode "flux" (default)
    or "diffusivity".  Returns per-member profile series at the snapshot steps."""
    ens = ocn.Ensemble(members)
    ens.set_mode("batched")        # coarse instances are small: one launch per kernel for all of them
    for p, m, st in zip(members, ens.members, init_states):
        m.set(project=False, **st)
        if closure is not None:
            c = closure(p) if callable(closure) else closure
            net, mu, sigma, scale = c[:4]
            m.set_column_closure(net, mu, sigma, scale, p["N2"], mode=c[4] if len(c) > 4 else "flux")
    ens.autotune()
    n = _time_steps(t_end, dt)
    series = [[] for _ in members]
    for step in range(0, n + 1, every):
        if step > 0:
            ens.time_step(dt, every)
        ens.synchronize()
        for i, m in enumerate(ens.members):
            series[i].append((step * dt, m.profiles()))
    return ens, series


def profile_errors(p: dict, coarse_series, fine_series) -> dict:
    """Normalised RMS errors over the snapshot times after t = 0:
    b: ||<b>_c - <b>_f|| / ||<b>_f - <b>_f(0)||  (dz-weighted over levels),
    Fb: ||F_c - F_f|| / ||F_f|| of the total mean vertical buoyancy flux (interior faces)."""
    zf = np.asarray(p["z_faces"])
    dzc = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzf = np.diff(zc)
    nb = db = nf = df = 0.0
    b0 = fine_series[0][1]["b"]
    for (t, pc), (_, pf) in zip(coarse_series[1:], fine_series[1:]):
        db += float((dzc * (pc["b"] - pf["b"]) ** 2).sum())
        nb += float((dzc * (pf["b"] - b0) ** 2).sum())
        df += float((dzf * (pc["Fb"][1:-1] - pf["Fb"][1:-1]) ** 2).sum())
        nf += float((dzf * pf["Fb"][1:-1] ** 2).sum())
    return {"b": math.sqrt(db / max(nb, 1e-300)), "Fb": math.sqrt(df / max(nf, 1e-300))}


def closure_for(net, mu, sigma, scale, yscale=None, mode="flux"):
    """The per-member closure arguments: with yscale "Jb" the output scales carry the member's
    surface buoyancy flux."""
    if yscale == "Jb":
        return lambda q: (net, mu, sigma, np.asarray(scale) * q["top_flux"]["b"], mode)
    return (net, mu, sigma, scale, mode)


def apriori_errors(pred, Y, G, n_members, Nz_of, cy, cx):
    """Normalised RMS error of the horizontal-mean predicted flux against the horizontal-mean
    target, per member (over faces and snapshots), for each flux component."""
    import torch
    out = np.zeros((n_members, 3))
    for i in range(n_members):
        sel = G == i
        if not bool(sel.any()):
            continue
        n_col = cx * cy
        Pm = pred[sel].reshape(-1, n_col, 3).mean(dim=1)
        Ym = Y[sel].double().reshape(-1, n_col, 3).mean(dim=1)
        out[i] = (torch.linalg.norm(Pm - Ym, dim=0) / torch.linalg.norm(Ym, dim=0).clamp_min(1e-300)).cpu().numpy()
    return out


def experiment(n_members: int = 64, n_train: int = 48, t_end: float = 6 * 3600.0, dt: float = 10.0,
               every: int = 180, cx: int = 16, cy: int = 16, train_steps: int = 3000, batch: int = 16384,
               lr: float = 1e-3, sizes=(64, 96, 128), depths=(64, 80, 96), variants=None, log=print) -> dict:
    """The learned-vs-plain comparison.  variants: {name: dict(target="column"|"mean",
    outputs=(0, 1, 2))}; each is trained on the training members and run on every member.
    Returns per-member errors and summaries over the held-out members."""
    import torch
    if variants is None:
        variants = {"mlp": DEFAULT_VARIANT, "cfg5": DIFFUSIVITY_VARIANT}
    members = inputs.ensemble_configs(n=n_members, sizes=sizes, depths=depths, dt=dt)
    coarse_members = [coarse_config(p, cx, cy) for p in members]
    t0 = time.time()
    coarse_feat = ocn.Ensemble(coarse_members)
    data = {t: ([], [], []) for t in set(v.get("target", "mean") for v in variants.values())}
    init_states = [None] * n_members

    def snapshot(step, ens):
        if step == 0:
            for i, m in enumerate(ens.members):
                c = m.coarse_grain(cx, cy)
                init_states[i] = {k: c[k].clone() for k in ("u", "v", "w", "b")}
            return
        for tgt, (Xs, Ys, Gs) in data.items():
            X, Y, G = training_samples(members, coarse_feat.members, ens, cx, cy, target=tgt)
            Xs.append(X); Ys.append(Y); Gs.append(G)

    fine, fine_series = fine_run(members, t_end, dt, every, cx, cy, on_snapshot=snapshot)
    torch.cuda.synchronize()
    t_fine = time.time() - t0
    del fine
    _, plain = coarse_run(coarse_members, init_states, t_end, dt, every, None)
    rows = [{"member": i, "train": i < n_train, "Nx": p["Nx"], "Nz": p["Nz"], "Jb": p["top_flux"]["b"], "N2": p["N2"],
             "f": p["f"]} for i, p in enumerate(members)]
    for i, p in enumerate(members):
        e = profile_errors(p, plain[i], fine_series[i])
        rows[i]["amd_b"], rows[i]["amd_Fb"] = e["b"], e["Fb"]
    summary = {"n_members": n_members, "n_train": n_train, "t_end": t_end, "dt": dt, "fine_seconds": t_fine}
    test = [i for i in range(n_members) if i >= n_train]
    summary["amd_b"] = float(np.mean([rows[i]["amd_b"] for i in test]))
    summary["amd_Fb"] = float(np.mean([rows[i]["amd_Fb"] for i in test]))
    nets = {}
    for name, v in variants.items():
        Xs, Ys, Gs = data[v.get("target", "mean")]
        X, Y, G = torch.cat(Xs), torch.cat(Ys), torch.cat(Gs)
        tr = G < n_train
        t1 = time.time()
        outputs = tuple(v.get("outputs", (0, 1, 2)))
        feats = {"nonlocal": NONLOCAL, "local": LOCAL}.get(v.get("features"))
        jb = torch.tensor([p["top_flux"]["b"] for p in members], dtype=torch.float64, device=X.device)
        ysc = None
        if v.get("scale") == "Jb":
            ysc = jb[G.long()][:, None].expand(-1, 3).contiguous()
        diffusive = v.get("form") == "diffusivity"
        Yt, wts = (diffusivity_targets(X, Y, cx * cy, v.get("kmax", KAPPA_MAX)) if diffusive else (Y, None))
        if v.get("weighting", "gradient") == "uniform":
            wts = None
        net, mu, sigma, scale, hist = train(X[tr], Yt[tr], steps=train_steps, batch=batch, lr=lr, outputs=outputs,
                                            features=feats, yscale=None if ysc is None else ysc[tr],
                                            weights=None if wts is None else wts[tr])
        t_train = time.time() - t1
        pred = predict(net, mu, sigma, scale, X)
        if ysc is not None:
            pred = pred * ysc
        if diffusive:        # the fluxes -K dq/dz of the predicted diffusivities, column by column
            K = pred.clamp_min(0.0)
            g3 = X[:, [2, 7, 12]].double()
            pred = torch.stack([-K[:, 0] * g3[:, 0], -K[:, 1] * g3[:, 1], -K[:, 1] * g3[:, 2]], dim=1)
        # a priori skill against the column-mean target of every member
        Xm, Ym, Gm = data["mean"] if "mean" in data else (Xs, Ys, Gs)
        ap = apriori_errors(pred, torch.cat(Ym), torch.cat(Gm), n_members, None, cy, cx)
        closure_fn = closure_for(net, mu, sigma, scale, v.get("scale"), "diffusivity" if diffusive else "flux")
        _, learned = coarse_run(coarse_members, init_states, t_end, dt, every, closure_fn)
        for i, p in enumerate(members):
            e = profile_errors(p, learned[i], fine_series[i])
            rows[i][f"{name}_b"], rows[i][f"{name}_Fb"] = e["b"], e["Fb"]
            rows[i][f"{name}_apriori_b"] = float(ap[i, 0])
        summary[f"{name}_b"] = float(np.mean([rows[i][f"{name}_b"] for i in test]))
        summary[f"{name}_Fb"] = float(np.mean([rows[i][f"{name}_Fb"] for i in test]))
        summary[f"{name}_apriori_b"] = float(np.mean([rows[i][f"{name}_apriori_b"] for i in test]))
        summary[f"{name}_loss"] = [float(hist[0]), float(np.mean(hist[-50:]))]
        summary[f"{name}_samples"] = int(tr.sum())
        summary[f"{name}_train_seconds"] = t_train
        nets[name] = (net, mu, sigma, scale, v.get("scale"), "diffusivity" if diffusive else "flux")
        log(f"{name}: loss {hist[0]:.4f} -> {np.mean(hist[-50:]):.4f} ({t_train:.1f} s); test b {summary[name + '_b']:.3f} "
            f"Fb {summary[name + '_Fb']:.3f} apriori {summary[name + '_apriori_b']:.3f} | amd b {summary['amd_b']:.3f} "
            f"Fb {summary['amd_Fb']:.3f}")
    return {"rows": rows, "summary": summary, "nets": nets}


class _Sub:
    """The first n members of an ensemble (training members only)."""

    def __init__(self, ens, n):
        self.members = ens.members[:n]


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned column closure vs plain AMD on coarse CBL runs")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--train", type=int, default=48)
    ap.add_argument("--hours", type=float, default=6.0)
    ap.add_argument("--dt", type=float, default=10.0)
    ap.add_argument("--every", type=int, default=180)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--rows", action="store_true", help="print every member's errors")
    a = ap.parse_args(argv)
    res = experiment(n_members=a.members, n_train=a.train, t_end=a.hours * 3600.0, dt=a.dt, every=a.every,
                     train_steps=a.steps, batch=a.batch)
    if a.rows:
        for r in res["rows"]:
            print(json.dumps({k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in r.items()}))
    print(json.dumps(res["summary"]))


if __name__ == "__main__":
    main()
