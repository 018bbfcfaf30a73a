"""What the trained network gains: relaxations of held-out bilayer points from its proposals
need fewer steps than from random starts, and reach the same state at the same tolerance."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_warm_start_saves_steps_and_reaches_the_same_state():
    from paper_2605_28800_b300 import tdgl, warmstart
    ctx = tdgl.Context(0)
    try:
        cfg = synth.CONFIG5
        pts = synth.bilayer_points(512 + 32, cfg["seed"], cfg["T"], cfg["Ez"], cfg["ratio"], cfg["shape"][2])
        rep = warmstart.run(ctx, cfg, pts, lambda shape, p: synth.uniform_P(shape, cfg["amp"], p["seed"]),
                            n_train=512, n_test=32, epochs=12, max_steps=20000, log=None)
    finally:
        ctx.close()
    assert rep["train_losses"][-1] < 0.05 * rep["train_losses"][0]
    # Training is reproducible from the seed.  With this budget (512 textures, 12 epochs) the
    # proposals save 10.6 % of the steps over the 32 held-out points and help at 30 of them; the
    # bounds leave room for changes of rounding in the solver.  Larger budgets save more (the
    # bench's 1800-texture run: about a quarter).
    assert rep["steps_saved_fraction_with_fallback"] > 0.05, rep["steps_saved_fraction_with_fallback"]
    assert rep["proposal_helped"] > 0.75
    assert rep["warm_converged"] >= 0.9
    # same tolerance, same state: energies and textures of the two relaxations agree
    assert rep["dF_rel_max_both_converged"] < 1e-6
    assert rep["texture_rms_rel_median"] < 1e-3
    # the single-simulation path and the batch take identical steps from the same start
    assert rep["sequential_equals_batched_steps"]


def test_rolling_batch_relaxation_matches_each_sim_alone():
    # the batched relaxation refills finished members' slots between slices; every point still
    # stops at the same step, in the same state, as when it relaxes alone (small grids, two slots,
    # 64-step slices: many refills and restarts)
    from paper_2605_28800_b300 import tdgl, warmstart
    ctx = tdgl.Context(0)
    try:
        cfg = dict(synth.CONFIG5, shape=(16, 16, 8))
        pts = synth.bilayer_points(7, 11, cfg["T"], cfg["Ez"], cfg["ratio"], cfg["shape"][2])
        starts = [synth.uniform_P(cfg["shape"], cfg["amp"], p["seed"]) for p in pts]
        seq = warmstart.relax_points(ctx, cfg, pts, starts, 1500, sequential=True)
        rol = warmstart.relax_points(ctx, cfg, pts, starts, 1500, chunk=2, slice_steps=64)
        # the state report of one batch call: converged members and members at the cap
        sims = [warmstart.make_sim(ctx, cfg["shape"], cfg["cell"], p, cfg["eps_b"], P) for p, P in zip(pts, starts)]
        b = tdgl.Batch(ctx, sims)
        ran, state = b.relax_state([cfg["dt_star"] / s.scales()[1] for s in sims], cfg["tol"], 1500)
        b.close()
        for s in sims:
            s.close()
    finally:
        ctx.close()
    P_seq, st_seq, cv_seq, F_seq = seq
    P_rol, st_rol, cv_rol, F_rol = rol
    assert st_rol == st_seq and cv_rol == cv_seq
    assert ran == st_seq
    assert state == [tdgl.RELAX_CONVERGED if c else tdgl.RELAX_AT_CAP for c in cv_seq]
    for a, b_ in zip(P_rol, P_seq):
        assert np.array_equal(a, b_)
    assert F_rol == F_seq
    assert 0 < sum(cv_seq)
