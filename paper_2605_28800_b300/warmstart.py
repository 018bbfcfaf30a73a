"""Learned warm start for the relaxation of PbTiO3/SrTiO3 bilayers.

The solver makes its own training data: seeded (T, Ez, layer thickness) points are relaxed from
random starts to the convergence tolerance (batched, one launch per kernel family), a 3D U-Net on
the tensor cores (tdgl.UNet) learns the map from per-cell inputs to the relaxed texture, and for a
new point its proposal replaces the random start.  The plain relaxation to the same tolerance then
judges the proposal: steps, final free energy and texture against the relaxation from the random
start, with the random start kept whenever the proposal does not save steps.

Everything numeric runs in libtdgl's kernels; this module only builds inputs, batches the calls
and keeps the books.  The caller supplies the (T, Ez, thickness) points and the random starts.
"""
from __future__ import annotations

import time

import numpy as np

from . import tdgl
from .materials import PTO, STO

#: scale of the network's output: the spontaneous polarization of PbTiO3 at 300 K (C/m^2)
P_SCALE = 0.7583600
T_MID, T_HALF = 300.0, 50.0
E_HALF = 1.5e8
N_IN, N_OUT = 4, 3


def bilayer_map(shape, t_pto) -> np.ndarray:
    """uint8 material map (nz, ny, nx): SrTiO3 (id 2) below, PbTiO3 (id 1) in the top t_pto layers."""
    nx, ny, nz = shape
    m = np.full((nz, ny, nx), 2, np.uint8)
    m[nz - t_pto:] = 1
    return m


def features(shape, point) -> np.ndarray:
    """Network input (4, nz, ny, nx): PbTiO3 and SrTiO3 indicators, (T - 300 K) / 50 K,
    Ez / 150 MV/m."""
    nx, ny, nz = shape
    m = bilayer_map(shape, point["t_pto"])
    f = np.empty((N_IN, nz, ny, nx), np.float32)
    f[0] = m == 1
    f[1] = m == 2
    f[2] = (point["T"] - T_MID) / T_HALF
    f[3] = point["Ez"] / E_HALF
    return f


def make_sim(ctx, shape, cell, point, eps_b, P):
    s = tdgl.Sim(ctx, shape, cell)
    s.define_material(1, PTO)
    s.define_material(2, STO)
    s.set_material_map(bilayer_map(shape, point["t_pto"]))
    s.set_eps_b(eps_b)
    s.set_temperature(point["T"])
    s.set_field((0.0, 0.0, point["Ez"]))
    s.set_P(P)
    return s


def relax_points(ctx, cfg, points, starts, max_steps, chunk=64, sequential=False, slice_steps=1024):
    """Relax every point from its start.  Returns the final textures (3, nz, ny, nx) float32, the
    steps taken, whether each converged, and the total energies.

    Batched: at most `chunk` sims at a time, relaxed in slices of `slice_steps` steps (a multiple of
    the 16-step check interval, so each sim is checked on the same steps as in one uninterrupted
    relaxation and stops at the same step).  Between slices the sims that finished (converged, or
    at max_steps) leave and the next points take their slots, so the batch stays full instead of
    waiting for its slowest member.  Sequential: each sim alone on the single-simulation path."""
    shape, cell = cfg["shape"], cfg["cell"]
    n = len(points)
    P_out, steps, conv, F = [None] * n, [0] * n, [False] * n, [None] * n

    def finish(i, s, converged):
        P_out[i] = s.get_P()
        conv[i] = bool(converged)
        F[i] = s.energy()["total"]
        s.close()

    if sequential:
        for i0 in range(0, n, chunk):
            sims = [make_sim(ctx, shape, cell, p, cfg["eps_b"], P) for p, P in zip(points[i0:i0 + chunk], starts[i0:i0 + chunk])]
            for j, s in enumerate(sims):
                k = s.relax(cfg["dt_star"] / s.scales()[1], cfg["tol"], max_steps, raise_on_cap=False)[0]
                steps[i0 + j] = int(k)
                finish(i0 + j, s, int(k) < max_steps)
        return P_out, steps, conv, F
    if slice_steps % 16:
        raise ValueError("slice_steps must be a multiple of the 16-step check interval")
    queue, active = list(range(n)), []
    while queue or active:
        while queue and len(active) < chunk:
            i = queue.pop(0)
            s = make_sim(ctx, shape, cell, points[i], cfg["eps_b"], starts[i])
            active.append((i, s, cfg["dt_star"] / s.scales()[1]))
        k = min(slice_steps, min(max_steps - steps[i] for i, _, _ in active))
        b = tdgl.Batch(ctx, [s for _, s, _ in active])
        ran, state = b.relax_state([dt for _, _, dt in active], cfg["tol"], k)
        b.close()
        keep = []
        for (i, s, dt), r, st in zip(active, ran, state):
            steps[i] += r
            if st in (tdgl.RELAX_DIVERGED, tdgl.RELAX_TIMEOUT):
                raise tdgl.TdglError(tdgl.EDIVERGED if st == tdgl.RELAX_DIVERGED else tdgl.ETIMEOUT,
                                     f"point {i} did not relax")
            if st == tdgl.RELAX_CONVERGED or steps[i] >= max_steps:
                finish(i, s, st == tdgl.RELAX_CONVERGED)
            else:
                keep.append((i, s, dt))
        active = keep
    return P_out, steps, conv, F


def train(net, X, Y, epochs, batch, lr, seed=0, log=None):
    """Adam on (X, Y) pairs (lists of (4, ...) inputs and (3, ...) targets scaled by P_SCALE),
    shuffled each epoch with a seeded generator; lr follows a cosine from lr down to lr / 20 over the
    run, so the last epochs average out the minibatch noise instead of ending on one of its swings.
    The pairs are moved to device memory once and batches are gathered there."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = torch.from_numpy(np.stack(X)).to(dev)
    Yd = torch.from_numpy(np.stack(Y).astype(np.float32)).to(dev)
    g = np.random.Generator(np.random.Philox(seed))
    n = len(X)
    steps_total = epochs * (n // batch)
    k = 0
    losses = []
    for ep in range(epochs):
        order = torch.from_numpy(g.permutation(n)).to(dev)
        run = []
        for j in range(0, n - batch + 1, batch):
            idx = order[j:j + batch]
            xb = Xd.index_select(0, idx).contiguous()
            yb = Yd.index_select(0, idx).contiguous()
            torch.cuda.current_stream().synchronize()     # the library runs on its own stream
            lr_k = lr * (0.05 + 0.475 * (1.0 + np.cos(np.pi * k / max(steps_total, 1))))
            run.append(net.train_step(xb, yb, lr_k))
            k += 1
        losses.append(float(np.mean(run)))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {losses[-1]:.5f}")
    del Xd, Yd
    return losses


P_CLIP = 1.25   # largest proposed |P_i| in units of P_SCALE


def propose(net, shape, points, batch):
    """Warm starts (3, nz, ny, nx) float32 in C/m^2 for the points.  Each component is clipped to
    +-P_CLIP P_SCALE: the relaxed textures of these bilayers stay below it, so a useful proposal is
    unchanged, while an untrained or badly trained network's outliers (the explicit step is unstable
    from polarizations far above saturation) cannot make the judging relaxation diverge."""
    out = []
    for i in range(0, len(points), batch):
        xb = np.stack([features(shape, p) for p in points[i:i + batch]])
        y = np.clip(net.forward(xb), -P_CLIP, P_CLIP)
        out.extend([(P_SCALE * y[j]).astype(np.float32) for j in range(y.shape[0])])
    return out


def conv_flops(shape, cin, cout, chans):
    """(forward, training) multiply-add flops per sample of the U-Net: 2 V Co Ci taps per
    convolution for the forward pass; training adds the data gradient (every layer but the first)
    and the weight gradient, each the same count."""
    nx, ny, nz = shape
    fwd = train = 0
    c_prev = cin
    layers = []
    for l, c in enumerate(chans):
        layers += [(l, c_prev, c, 27, l > 0), (l, c, c, 27, True)]
        c_prev = c
    for l in range(len(chans) - 2, -1, -1):
        layers += [(l, c_prev + chans[l], chans[l], 27, True), (l, chans[l], chans[l], 27, True)]
        c_prev = chans[l]
    layers.append((0, chans[0], cout, 1, True))
    for l, ci, co, taps, dx in layers:
        v = (nx >> l) * (ny >> l) * (nz >> l)
        f = 2.0 * v * ci * co * taps
        fwd += f
        train += f * (3 if dx else 2)
    return fwd, train


def texture_distance(Pa, Pb):
    """RMS difference of two textures relative to the RMS of the second"""
    return float(np.sqrt(np.mean((Pa - Pb) ** 2)) / max(np.sqrt(np.mean(Pb ** 2)), 1e-30))


def run(ctx, cfg, points, random_start, n_train, n_test, epochs, max_steps, batch=4, lr=2e-3,
        chans=(16, 32, 64, 128), log=print):
    """The whole protocol: generate, train, judge.  cfg: shape, cell, eps_b, dt_star, tol, seed;
    points: at least n_train + n_test dicts with T, Ez, t_pto (PbTiO3 layers on top); random_start
    (shape, point) -> the float32 (3, nz, ny, nx) random start of a point.  The first n_train points
    train, the next n_test are held out.  Returns a report dict."""
    log = log or (lambda m: None)
    shape = cfg["shape"]
    if len(points) < n_train + n_test:
        raise ValueError("fewer points than n_train + n_test")
    train_pts, test_pts = points[:n_train], points[n_train:n_train + n_test]
    t0 = time.perf_counter()
    P_tr, st_tr, cv_tr, _ = relax_points(ctx, cfg, train_pts, [random_start(shape, p) for p in train_pts],
                                         max_steps)
    t_gen = time.perf_counter() - t0
    log(f"generated {n_train} relaxed textures in {t_gen:.1f} s (median {np.median(st_tr):.0f} steps, "
        f"{np.mean(cv_tr):.2f} converged)")
    X = [features(shape, p) for p in train_pts]
    Y = [P / P_SCALE for P in P_tr]
    net = tdgl.UNet(ctx, shape, N_IN, N_OUT, chans=chans, max_batch=batch, seed=cfg["seed"])
    t0 = time.perf_counter()
    losses = train(net, X, Y, epochs, batch, lr, seed=cfg["seed"], log=log)
    t_train = time.perf_counter() - t0
    # judge on held-out points at the same tolerance and dt: plain (each sim alone, random start),
    # batched (random start) and batched from the network's proposals
    rnd = [random_start(shape, p) for p in test_pts]
    t0 = time.perf_counter()
    P_seq, st_seq, cv_seq, F_seq = relax_points(ctx, cfg, test_pts, rnd, max_steps, sequential=True)
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    P_plain, st_plain, cv_plain, F_plain = relax_points(ctx, cfg, test_pts, rnd, max_steps)
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    starts = propose(net, shape, test_pts, batch)
    t_inf = time.perf_counter() - t0
    t0 = time.perf_counter()
    P_warm, st_warm, cv_warm, F_warm = relax_points(ctx, cfg, test_pts, starts, max_steps)
    t_warm = time.perf_counter() - t0
    st_plain, st_warm = np.array(st_plain), np.array(st_warm)
    chosen = np.minimum(st_plain, st_warm)          # random start kept when the proposal does not help
    dF = np.array(F_warm) - np.array(F_plain)
    f_fwd, f_train = conv_flops(shape, N_IN, N_OUT, chans)
    n_steps = epochs * (n_train // batch)
    return dict(
        conv_gflop_per_sample_forward=f_fwd / 1e9, conv_gflop_per_sample_training=f_train / 1e9,
        train_tflops=f_train * batch * n_steps / max(t_train, 1e-9) / 1e12,
        infer_tflops=f_fwd * n_test / max(t_inf, 1e-9) / 1e12,
        n_train=n_train, n_test=n_test, epochs=epochs, batch=batch, lr=lr, chans=list(chans),
        params=net.param_count(), max_steps=max_steps, tol=cfg["tol"],
        gen_seconds=t_gen, train_seconds=t_train, infer_seconds=t_inf,
        train_loss_first=losses[0], train_loss_last=losses[-1], train_losses=losses,
        train_steps_median=float(np.median(st_tr)), train_converged=float(np.mean(cv_tr)),
        relaxed_P_abs_max=float(max(float(np.abs(P).max()) for P in P_tr)), proposal_clip=P_CLIP * P_SCALE,
        plain_steps=st_plain.tolist(), warm_steps=st_warm.tolist(),
        plain_steps_total=int(st_plain.sum()), warm_steps_total=int(st_warm.sum()),
        steps_saved_fraction=float(1.0 - st_warm.sum() / max(st_plain.sum(), 1)),
        proposal_helped=float(np.mean(st_warm < st_plain)),
        # the same, over the points whose plain relaxation converged within max_steps
        steps_saved_fraction_plain_converged=float(
            1.0 - st_warm[np.array(cv_plain)].sum() / max(st_plain[np.array(cv_plain)].sum(), 1)),
        dF_rel_max_plain_converged=float(np.max((np.abs(dF) / np.maximum(np.abs(np.array(F_plain)), 1e-300))
                                                [np.array(cv_plain)])) if any(cv_plain) else None,
        dF_rel_max_both_converged=float(np.max((np.abs(dF) / np.maximum(np.abs(np.array(F_plain)), 1e-300))
                                               [np.array(cv_plain) & np.array(cv_warm)]))
        if any(np.array(cv_plain) & np.array(cv_warm)) else None,
        # the protocol: the proposal where it saves steps, else the random start
        steps_saved_fraction_with_fallback=float(1.0 - chosen.sum() / max(st_plain.sum(), 1)),
        with_fallback_steps_total=int(chosen.sum()),
        sequential_plain_seconds=t_seq, batched_plain_seconds=t_plain, batched_warm_seconds=t_warm + t_inf,
        speedup_vs_sequential_plain=float(t_seq / max(t_warm + t_inf, 1e-9)),
        speedup_vs_batched_plain=float(t_plain / max(t_warm + t_inf, 1e-9)),
        sequential_equals_batched_steps=bool(np.array_equal(np.array(st_seq), st_plain)),
        plain_converged=float(np.mean(cv_plain)), warm_converged=float(np.mean(cv_warm)),
        dF_rel_median=float(np.median(np.abs(dF) / np.maximum(np.abs(np.array(F_plain)), 1e-300))),
        dF_rel_max=float(np.max(np.abs(dF) / np.maximum(np.abs(np.array(F_plain)), 1e-300))),
        texture_rms_rel_median=float(np.median([texture_distance(a, b) for a, b in zip(P_warm, P_plain)])),
        proposal_rms_rel_median=float(np.median([texture_distance(a, b) for a, b in zip(starts, P_plain)])),
    )
