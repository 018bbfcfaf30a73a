"""Runtime behaviour of the CUDA path through the C ABI: batches, relaxation, random start,
edge cases and error codes (no GPU fault is provoked: every bad input is rejected on the host)."""
import numpy as np
import pytest

import synth
from oracle import coefficients
from tests.helpers import gpu_sim, oracle_sys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    yield c
    c.close()


def _bto(ctx, shape, T=300.0, seed=1, eps_b=45.0):
    nx, ny, nz = shape
    mat = np.ones((nz, ny, nx), np.uint8)
    P = synth.uniform_P(shape, 0.01, seed)
    return gpu_sim(ctx, shape, (1e-9,) * 3, mat, {1: synth.BTO}, T, eps_b, P=P), P


@pytest.mark.parametrize("nsteps", [7, 16])
def test_batch_equals_single_runs_bitwise(ctx, nsteps):
    # odd counts run launch by launch, even counts replay captured graphs
    from paper_2605_28800_b300 import tdgl
    shapes = [(16, 16, 16), (12, 20, 8), (9, 7, 5), (32, 8, 4)]
    temps = [300.0, 250.0, 350.0, 200.0]
    dt = [0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"]) * f for f in (1.0, 0.8, 1.2, 0.5)]
    singles, batched = [], []
    for i, (sh, T) in enumerate(zip(shapes, temps)):
        a, _ = _bto(ctx, sh, T, seed=10 + i)
        b, _ = _bto(ctx, sh, T, seed=10 + i)
        singles.append(a)
        batched.append(b)
    for a, d in zip(singles, dt):
        a.step(nsteps, d)
        a.energy()
        a.step(nsteps, d)
    B = tdgl.Batch(ctx, batched)
    B.step(nsteps, dt)
    for b in batched:
        b.energy()
    B.step(nsteps, dt)
    for a, b in zip(singles, batched):
        assert np.array_equal(a.get_P(), b.get_P())
    B.close()


def test_batch_members_match_oracle(ctx):
    # every member of a ragged batch (radix-2 and radix-3 transform lengths, the 48^3 member of the
    # uneven sweep among them) against the FP64 oracle run of the same sim: 8 batched steps, an
    # energy call on each member (it leaves the field spectrum for the next step), 8 more steps
    from paper_2605_28800_b300 import tdgl
    members = [((16, 16, 16), 300.0, 1.0), ((12, 20, 8), 250.0, 0.8), ((48, 48, 48), 300.0, 1.0),
               ((96, 24, 8), 200.0, 0.5), ((9, 7, 5), 350.0, 1.2), ((40, 16, 8), 300.0, 1.0)]
    a1 = abs(coefficients(synth.BTO, 300.0)["a1x"])
    sims, starts, dts = [], [], []
    for i, (sh, T, f) in enumerate(members):
        nx, ny, nz = sh
        P = synth.uniform_P(sh, 0.15, 40 + i)
        sims.append(gpu_sim(ctx, sh, (1e-9,) * 3, np.ones((nz, ny, nx), np.uint8), {1: synth.BTO}, T, 45.0, P=P))
        starts.append(P)
        dts.append(0.004 / a1 * f)
    B = tdgl.Batch(ctx, sims)
    B.step(8, dts)
    for s in sims:
        s.energy()
    B.step(8, dts)
    for (sh, T, _), s, P, dt in zip(members, sims, starts, dts):
        nx, ny, nz = sh
        o = oracle_sys(sh, (1e-9,) * 3, np.ones((nz, ny, nx), np.uint8), {1: synth.BTO}, T, 45.0)
        want = o.run(P.astype(np.float64), dt, 16)
        got = s.get_P()
        moved = np.abs(want - P).max()
        err = np.abs(got - want).max()
        assert err / s.scales()[0] <= 1e-5, (sh, err)
        assert err <= 1e-3 * moved, (sh, err, moved)
    B.close()


def test_batch_relax_converged_sims_leave_the_work_list(ctx):
    from paper_2605_28800_b300 import tdgl
    sims = []
    for i, T in enumerate((300.0, 420.0)):
        s, _ = _bto(ctx, (8, 8, 8), T, seed=20 + i)
        sims.append(s)
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    B = tdgl.Batch(ctx, sims)
    steps, ok = B.relax(dt, 1e-6, 200000, check_every=16)
    assert ok
    assert steps[0] != steps[1]
    for s in sims:
        # each sim satisfies the criterion on its own after the batch stopped it
        s.step(1, dt)
        assert s.last_max_dP() < 1.5e-6
    B.close()


@pytest.mark.parametrize("max_steps", [4000, 1208])
def test_batch_device_relax_equals_single_relaxations(ctx, max_steps):
    # the batch's device loop retires members as they converge (their kernels' blocks return at
    # once) and hands back to the host to rebuild the work lists; every member must stop at the
    # same step, in the same state, as its own relaxation (1208: a cap that is not a multiple of the
    # check interval, finished by host-checked chunks)
    from paper_2605_28800_b300 import tdgl
    shapes = [(16, 16, 16), (12, 20, 8), (24, 24, 24), (9, 7, 5), (32, 16, 8)]
    temps = [420.0, 300.0, 440.0, 410.0, 300.0]
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    singles, members = [], []
    for i, (sh, T) in enumerate(zip(shapes, temps)):
        a, _ = _bto(ctx, sh, T, seed=60 + i)
        b, _ = _bto(ctx, sh, T, seed=60 + i)
        singles.append(a)
        members.append(b)
    want = [s.relax(dt, 1e-6, max_steps, check_every=16, raise_on_cap=False)[0] for s in singles]
    B = tdgl.Batch(ctx, members)
    got, _ = B.relax(dt, 1e-6, max_steps, check_every=16, raise_on_cap=False)
    assert list(got) == list(want)
    assert min(want) < max_steps and max(want) <= max_steps
    for a, b in zip(singles, members):
        assert np.array_equal(a.get_P(), b.get_P())
        assert b.last_max_dP() == a.last_max_dP()
    B.close()


def test_row_tile_autotuner_times_candidates_and_reuses_the_choice():
    # the first preparation of a sim shape times each candidate tile of the step kernel on scratch
    # buffers (state unchanged) and keeps the fastest for the context; a second sim of the shape
    # reuses it, and both step like the oracle
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    try:
        shape = (32, 32, 16)
        dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
        a, P = _bto(c, shape, seed=71)
        assert a.row_tile()[0] == 0
        a.step(2, dt)
        tile, cands = a.row_tile()
        assert len(cands) >= 2 and all(us > 0 for _, us in cands)
        assert tile == min(cands, key=lambda cu: cu[1])[0]
        b, _ = _bto(c, shape, seed=71)
        b.step(2, dt)
        assert b.row_tile() == (tile, cands)
        assert np.array_equal(a.get_P(), b.get_P())
        nx, ny, nz = shape
        o = oracle_sys(shape, (1e-9,) * 3, np.ones((nz, ny, nx), np.uint8), {1: synth.BTO}, 300.0, 45.0)
        assert np.abs(a.get_P() - o.run(P.astype(np.float64), dt, 2)).max() / a.scales()[0] <= 1e-5
    finally:
        c.close()


def test_forced_row_tile_steps_like_the_tuned_one():
    # a sim whose row tile is forced (before its first step, and again after its step graphs were
    # captured) reports that tile, clamped to the kernel's maximum, and steps like the tuned sim
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    try:
        shape = (32, 32, 16)
        dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
        a, P = _bto(c, shape, seed=73)
        a.step(40, dt)
        f, _ = _bto(c, shape, seed=73)
        f.set_row_tile(2)
        f.step(20, dt)
        assert f.row_tile() == (2, [])
        f.set_row_tile(1000)                  # after the step graphs were captured
        assert f.row_tile()[0] < 1000 and f.row_tile()[0] >= 2
        f.step(20, dt)
        assert np.abs(f.get_P() - a.get_P()).max() / a.scales()[0] <= 1e-6
        with pytest.raises(tdgl.TdglError):
            f.set_row_tile(-1)
        f.set_row_tile(0)                     # back to the tuner (its record for this shape)
        f.step(2, dt)
        a.step(2, dt)
        assert f.row_tile()[0] == a.row_tile()[0]
    finally:
        c.close()


def test_fft_padding_defaults_and_forced_lengths(ctx):
    # defaults: smallest 2^a 3^b >= 2n - 1 (x even); z gives way to 128 / 256 / 512 within 4/3, y and z
    # to the smallest specialized length within 4/3, and x (rows a multiple of 4 long) to twice the
    # smallest specialized half-length >= nx within 4/3;
    # forced lengths are validated, and a sim re-padded between steps follows the same trajectory
    from paper_2605_28800_b300 import tdgl
    cases = {(96, 96, 96): (192, 192, 256), (48, 48, 48): (96, 96, 128), (17, 9, 5): (36, 18, 9),
             (32, 32, 8): (64, 64, 16), (128, 128, 128): (256, 256, 256),
             (40, 40, 81): (96, 96, 192),   # x: 81 is odd, so 96; y 81 and z 162 give way to 96 and 192
             (80, 80, 80): (192, 192, 192), (40, 40, 40): (96, 96, 96), (3, 5, 7): (6, 9, 16),
             (24, 20, 48): (64, 48, 128), (12, 20, 8): (32, 48, 16)}
    for shape, want in cases.items():
        s = tdgl.Sim(ctx, shape, (1e-9,) * 3)
        assert s.fft_pad() == want, shape
        s.close()
    a, P = _bto(ctx, (24, 20, 48), seed=97)
    b, _ = _bto(ctx, (24, 20, 48), seed=97)
    assert a.fft_pad()[2] == 128
    for bad in ((47, 0, 0), (48, 38, 0), (0, 0, 100), (0, 0, 64)):
        with pytest.raises(tdgl.TdglError) as e:
            b.set_fft_pad(*bad)
        assert e.value.code == tdgl.EINVAL
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    a.step(12, dt)
    b.step(6, dt)
    b.set_fft_pad(54, 0, 96)
    assert b.fft_pad() == (54, 48, 96)
    b.step(6, dt)
    b.set_fft_pad(0, 0, 0)
    assert b.fft_pad() == a.fft_pad()
    assert np.abs(a.get_P() - b.get_P()).max() / a.scales()[0] <= 1e-6


def test_async_host_io_pipeline_equals_synchronous_calls(ctx):
    # a queue of independent problems through the pipelined calls (upload, steps, download, no host
    # wait until sync) gives each problem the same P, bit for bit, as set_P / step / get_P; the
    # results match the oracle; sync reports divergence; RK45 is refused
    import torch
    from paper_2605_28800_b300 import tdgl
    shape = (32, 32, 16)
    nx, ny, nz = shape
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    s, _ = _bto(ctx, shape, seed=91)
    inputs = [torch.from_numpy(synth.uniform_P(shape, 0.05, 200 + k)).pin_memory() for k in range(5)]
    outs = [torch.full((3, nz, ny, nx), float("nan")).pin_memory() for _ in inputs]
    for Pin, Pout in zip(inputs, outs):
        s.set_P_async(Pin)
        s.step_async(3, dt)
        s.get_P_async(Pout)
    s.sync()
    for Pin, Pout in zip(inputs, outs):
        s.set_P(Pin.numpy())
        s.step(3, dt)
        assert np.array_equal(Pout.numpy(), s.get_P())
    o = oracle_sys(shape, (1e-9,) * 3, np.ones((nz, ny, nx), np.uint8), {1: synth.BTO}, 300.0, 45.0)
    want = o.run(inputs[-1].numpy().astype(np.float64), dt, 3)
    assert np.abs(outs[-1].numpy() - want).max() / s.scales()[0] <= 1e-5
    # continuing a sim: snapshots taken between queued steps
    s.set_P(inputs[0].numpy())
    snaps = [torch.empty(3, nz, ny, nx).pin_memory() for _ in range(3)]
    for snap in snaps:
        s.step_async(2, dt)
        s.get_P_async(snap)
    s.sync()
    s.set_P(inputs[0].numpy())
    for snap in snaps:
        s.step(2, dt)
        assert np.array_equal(snap.numpy(), s.get_P())
    # divergence of queued steps is reported by sync, and the sim is usable afterwards
    s.set_P_async(inputs[1])
    s.step_async(50, 1e-6)                  # far beyond the explicit stability bound
    with pytest.raises(tdgl.TdglError) as e:
        s.sync()
    assert e.value.code == tdgl.EDIVERGED
    s.set_P(inputs[1].numpy())
    s.step(3, dt)
    s.set_integrator(tdgl.RK45)
    with pytest.raises(tdgl.TdglError):
        s.step_async(1, dt)
    with pytest.raises(ValueError):
        s.get_P_async(torch.empty(3, nz, ny, nx, device="cuda"))


def test_bounded_wait_times_out_and_the_context_stays_usable(ctx):
    # a wait on an mbarrier that nothing will complete (no copy in flight) gives up after its poll
    # limit; the library reports ETIMEOUT and the same context keeps stepping correctly
    from paper_2605_28800_b300 import tdgl
    assert ctx.wait_probe(1000) == tdgl.ETIMEOUT
    assert "gave up" in ctx.last_error()
    assert ctx.wait_probe(0) == tdgl.EINVAL
    s, P = _bto(ctx, (8, 8, 4), seed=81)
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    s.step(3, dt)
    o = oracle_sys((8, 8, 4), (1e-9,) * 3, np.ones((4, 8, 8), np.uint8), {1: synth.BTO}, 300.0, 45.0)
    assert np.abs(s.get_P() - o.run(P.astype(np.float64), dt, 3)).max() / s.scales()[0] <= 1e-5


def test_relax_reaches_oracle_state(ctx):
    shape = (6, 6, 4)
    nx, ny, nz = shape
    mat = np.ones((nz, ny, nx), np.uint8)
    P = synth.uniform_P(shape, 0.01, 4)
    P[2] += 0.05
    # eps_B = 649 and a 50 MV/m field along z give a polarized, non-uniform relaxed state
    g = gpu_sim(ctx, shape, (1e-9,) * 3, mat, {1: synth.BTO}, 300.0, 649.0, E=(0.0, 0.0, 5e7), P=P)
    o = oracle_sys(shape, (1e-9,) * 3, mat, {1: synth.BTO}, 300.0, 649.0, E=(0.0, 0.0, 5e7))
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    n, ok = g.relax(dt, 1e-7, 400000, check_every=16)
    assert ok
    Po, no, oko = o.relax(P.astype(np.float64), dt, 1e-7, g.scales()[0], 400000, check_every=16)
    assert oko
    eg, eo = g.energy(), o.energy(Po)
    assert abs(eg["total"] - eo["total"]) <= 1e-5 * sum(abs(eo[k]) for k in ("land", "grad", "elec", "ext"))
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-3


def _philox_first(c, k):
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    c, k = list(c), list(k)
    for _ in range(10):
        p0, p1 = M0 * c[0], M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & 0xFFFFFFFF, p1 & 0xFFFFFFFF, ((p0 >> 32) ^ c[3] ^ k[1]) & 0xFFFFFFFF,
             p0 & 0xFFFFFFFF]
        k = [(k[0] + W0) & 0xFFFFFFFF, (k[1] + W1) & 0xFFFFFFFF]
    return c[0]


def test_philox_reference_known_answers():
    # known-answer vectors of Philox4x32-10 (Random123 distribution, kat_vectors): first word
    assert _philox_first([0, 0, 0, 0], [0, 0]) == 0x6627E8D5
    assert _philox_first([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == 0x408F276D
    assert _philox_first([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == 0xD16CFE09


def test_init_random_is_the_documented_philox_stream(ctx):
    shape = (7, 5, 3)
    s, _ = _bto(ctx, shape)
    seed, amp = 0x1234_5678_9ABC, 0.02
    s.init_random(seed, amp)
    P = s.get_P()
    ncell = 7 * 5 * 3
    want = np.empty(3 * ncell)
    for i in range(3 * ncell):
        u = _philox_first([i % ncell, i // ncell, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        want[i] = amp * (2.0 * ((u + 0.5) / 2 ** 32) - 1.0)
    assert np.allclose(P.ravel(), want, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 9), (9, 1, 1), (1, 7, 1), (3, 5, 7), (2, 2, 2)])
def test_degenerate_grids_step(ctx, shape):
    s, P = _bto(ctx, shape)
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    nx, ny, nz = shape
    o = oracle_sys(shape, (1e-9,) * 3, np.ones((nz, ny, nx), np.uint8), {1: synth.BTO}, 300.0, 45.0)
    s.step(20, dt)
    Po = o.run(P.astype(np.float64), dt, 20)
    assert np.abs(s.get_P() - Po).max() / s.scales()[0] <= 1e-5


def test_all_vacuum_map_keeps_zero(ctx):
    from paper_2605_28800_b300 import tdgl
    s = tdgl.Sim(ctx, (4, 4, 4), (1e-9,) * 3)
    s.define_material(1, synth.BTO)
    s.set_material_map(np.zeros((4, 4, 4), np.uint8))
    s.set_P(np.ones((3, 4, 4, 4), np.float32))
    s.step(3, 1e-12)
    assert np.all(s.get_P() == 0)


def test_invalid_arguments_are_rejected(ctx):
    from paper_2605_28800_b300 import tdgl
    with pytest.raises(tdgl.TdglError) as e:
        tdgl.Sim(ctx, (0, 4, 4), (1e-9,) * 3)
    assert e.value.code == tdgl.EINVAL
    with pytest.raises(tdgl.TdglError):
        tdgl.Sim(ctx, (tdgl.MAX_DIM + 1, 1, 1), (1e-9,) * 3)
    with pytest.raises(tdgl.TdglError):
        tdgl.Sim(ctx, (4, 4, 4), (1e-9, -1.0, 1e-9))
    s = tdgl.Sim(ctx, (4, 4, 4), (1e-9,) * 3)
    with pytest.raises(tdgl.TdglError):
        s.define_material(16, synth.BTO)
    with pytest.raises(tdgl.TdglError) as e:
        s.step(1, 1e-12)                       # no material defined
    assert e.value.code == tdgl.ESTATE
    s.define_material(1, synth.BTO)
    with pytest.raises(tdgl.TdglError):
        s.set_material_map(np.full((4, 4, 4), 20, np.uint8))
    m = np.ones((4, 4, 4), np.uint8); m[0, 0, 0] = 3   # undefined id
    s.set_material_map(m)
    with pytest.raises(tdgl.TdglError) as e:
        s.step(1, 1e-12)
    assert e.value.code == tdgl.ESTATE
    s.set_material_map(np.ones((4, 4, 4), np.uint8))
    with pytest.raises(tdgl.TdglError):
        s.step(1, -1.0)
    with pytest.raises(tdgl.TdglError):
        s.set_eps_b(0.0)
    with pytest.raises(tdgl.TdglError):
        s.set_temperature(-5.0)


def test_divergence_is_reported(ctx):
    from paper_2605_28800_b300 import tdgl
    s, _ = _bto(ctx, (6, 6, 6))
    with pytest.raises(tdgl.TdglError) as e:
        s.step(50, 1e-6)                       # far beyond the explicit stability bound
    assert e.value.code == tdgl.EDIVERGED


@pytest.mark.parametrize("integ", ["euler", "heun"])
@pytest.mark.parametrize("shape", [(16, 16, 16), (9, 7, 5)])
def test_device_relax_loop_matches_the_host_checked_loop(ctx, integ, shape):
    # tdgl_relax runs its convergence loop inside one CUDA graph (conditional while node) when
    # it can; with profiling on it checks on the host after every k steps.  Both take the same
    # steps to the same bits: to convergence, and to a step cap that is not a multiple of k
    from paper_2605_28800_b300 import tdgl
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    for tol, cap in ((1e-6, 400000), (1e-12, 100)):
        runs = []
        for host in (False, True):
            s, _ = _bto(ctx, shape, seed=23)
            if integ == "heun":
                s.set_integrator(tdgl.HEUN)
            ctx.profile(host)
            try:
                n, ok = s.relax(dt, tol, cap, check_every=16, raise_on_cap=False)
            finally:
                ctx.profile(False)
            runs.append((n, ok, s.get_P(), s.time()))
            s.close()
        (n0, ok0, P0, t0), (n1, ok1, P1, t1) = runs
        assert (n0, ok0) == (n1, ok1)
        assert ok0 == (cap > 1000)
        if cap == 100:
            assert n0 == 100
        assert np.array_equal(P0, P1)
        assert t0 == t1


def test_relax_after_an_energy_call_matches_the_host_checked_loop(ctx):
    # an energy call leaves the field spectrum of the current P; relax then runs its first chunk
    # host-checked (using that spectrum) and the rest in the device loop: same steps, same bits as
    # checking on the host throughout, across several relax / energy rounds
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    runs = []
    for host in (False, True):
        s, _ = _bto(ctx, (16, 16, 16), seed=29)
        ctx.profile(host)
        try:
            out = []
            for _ in range(3):
                e = s.energy()
                n, ok = s.relax(dt, 1e-12, 48, check_every=16, raise_on_cap=False)
                out.append((n, ok, e["total"]))
            out.append(s.get_P())
        finally:
            ctx.profile(False)
        runs.append(out)
        s.close()
    for a, b in zip(runs[0][:-1], runs[1][:-1]):
        assert a[:2] == b[:2]
        assert a[2] == pytest.approx(b[2], rel=1e-12)     # float64 block sums added in any order
    assert np.array_equal(runs[0][-1], runs[1][-1])


def test_device_relax_loop_reports_divergence(ctx):
    from paper_2605_28800_b300 import tdgl
    s, _ = _bto(ctx, (6, 6, 6))
    with pytest.raises(tdgl.TdglError) as e:
        s.relax(1e-6, 1e-6, 1000, check_every=16)    # far beyond the explicit stability bound
    assert e.value.code == tdgl.EDIVERGED
    assert "after 16 steps" in str(e.value)


def test_device_buffers_round_trip(ctx):
    import torch
    shape = (10, 6, 4)
    s, P = _bto(ctx, shape)
    Pt = torch.from_numpy(P).cuda()
    torch.cuda.synchronize()          # device buffers are read and written on the library's stream
    s.set_P(Pt)
    out = torch.empty_like(Pt)
    s.get_P(out)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), P, rtol=2e-7, atol=1e-12)


def test_launch_counter_counts_kernels(ctx):
    s, _ = _bto(ctx, (8, 8, 8))
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    s.step(1, dt)
    n0 = ctx.launch_count
    s.step(10, dt)
    assert ctx.launch_count - n0 == 10 * 4


@pytest.mark.parametrize("nz,length", [(128, 256), (64, 128)])
def test_zpass_autotuner_picks_a_variant_and_every_variant_agrees_with_the_oracle(nz, length):
    # 16 x 16 x 128 pads z to 256 points, 16 x 16 x 64 to 128: the context times the four
    # variants of the z pass on first use and keeps the fastest; forcing any of them gives the
    # same trajectory as the oracle
    from paper_2605_28800_b300 import tdgl
    from tests.helpers import mixed_case
    CELL = (1e-9, 1.1e-9, 0.9e-9)
    MATS = {1: synth.BTO, 2: dict(synth.PTO, G12=3e-11, G44=7e-11, G44p=2e-11)}
    shape = (16, 16, nz)
    mat, P = mixed_case(shape, seed=41)
    P *= 0.3
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    ctx = tdgl.Context(0)
    try:
        assert ctx.zpass_variant(length)[0] == -1
        finals = []
        for forced in (None, 0, 1, 2, 3):
            g = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, P=P)
            if forced is not None:
                ctx.set_zpass_variant(length, forced)
            g.step(3, dt)
            if forced is None:
                v, us = ctx.zpass_variant(length)
                assert len(us) == tdgl.ZPASS_VARIANTS == 4
                assert v in (0, 1, 2, 3) and min(us) > 0 and us[v] == min(us)
            else:
                assert ctx.zpass_variant(length)[0] == forced
            finals.append(g.get_P())
            g.close()
        o = oracle_sys(shape, CELL, mat, MATS, 300.0, 45.0)
        Po = o.run(P.astype(np.float64), dt, 3)
        for Pg in finals:
            assert np.abs(Pg - Po).max() / 0.2649096 <= 1e-5
        with pytest.raises(tdgl.TdglError):
            ctx.set_zpass_variant(64, 1)           # 64-point lines have one shape
        with pytest.raises(tdgl.TdglError):
            ctx.set_zpass_variant(512, 2)          # the staged variants exist for 128 and 256 only
        ctx.set_zpass_variant(512, 1)
    finally:
        ctx.close()


def test_fp32_fma_peak_is_plausible(ctx):
    # the probe reports between a tenth and 1.1 times the nominal FP32 rate of the device
    import torch
    p = torch.cuda.get_device_properties(0)
    nominal = p.multi_processor_count * 128 * 2 * 2.2e9 / 1e12       # 128 FP32 lanes per SM, <= 2.2 GHz
    v = ctx.fp32_fma_peak()
    assert 0.1 * nominal < v < 1.1 * nominal, (v, nominal)


def test_long_step_calls_run_as_bounded_chunks(ctx):
    # a step call longer than one chunk replays one cached 64-step graph per chunk (plus one for the
    # remainder): the same states, bit for bit, as the same steps in short calls, for a sim and a
    # batch; under an AC field (each chunk's phase from its own start time) the trajectory still
    # matches short calls to rounding
    from paper_2605_28800_b300 import tdgl
    shape = (16, 16, 8)
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    a, _ = _bto(ctx, shape, seed=61)
    b, _ = _bto(ctx, shape, seed=61)
    a.step(301, dt)
    for n in (50, 64, 1, 100, 86):
        b.step(n, dt)
    assert np.array_equal(a.get_P(), b.get_P())
    c, _ = _bto(ctx, shape, seed=62)
    d, _ = _bto(ctx, (12, 20, 8), seed=63)
    e, _ = _bto(ctx, shape, seed=62)
    f, _ = _bto(ctx, (12, 20, 8), seed=63)
    B = tdgl.Batch(ctx, [c, d])
    B.step(150, [dt, 0.8 * dt])
    B.close()
    for n in (40, 40, 40, 30):
        e.step(n, dt)
        f.step(n, 0.8 * dt)
    assert np.array_equal(c.get_P(), e.get_P()) and np.array_equal(d.get_P(), f.get_P())
    g, _ = _bto(ctx, shape, seed=64)
    h, _ = _bto(ctx, shape, seed=64)
    for s in (g, h):
        s.set_field_ac((0.0, 0.0, 5e7), 2e9)
    g.step(200, dt)
    for _ in range(10):
        h.step(20, dt)
    assert np.abs(g.get_P() - h.get_P()).max() <= 1e-6 * np.abs(h.get_P()).max()
    assert g.time() == pytest.approx(h.time(), rel=1e-12)
