"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: the fields are compared relative to the largest magnitude of the same field
(float32 arithmetic, FFT round-off grows like log N: 2e-5); trajectories use the stated bar
max|P_gpu - P_oracle| / P0 <= 1e-5 after 100 and 200 steps and |dF| / sum|F_terms| <= 1e-6.
"""
import numpy as np
import pytest

import synth
from oracle import coefficients
from oracle import tensor as otensor
from tests.helpers import gpu_sim, mixed_case, oracle_sys, rel_err

pytestmark = pytest.mark.gpu

CELL = (1e-9, 1.1e-9, 0.9e-9)
MATS = {1: synth.BTO, 2: dict(synth.PTO, G12=3e-11, G44=7e-11, G44p=2e-11, r_s=1.3)}
SHAPES = [(1, 1, 1), (1, 1, 6), (5, 1, 1), (3, 5, 7), (8, 8, 4), (17, 9, 5), (32, 32, 8), (24, 12, 20),
          # the transform lengths of the uneven sweep's 48^3 and 96^3 members, one axis at a time:
          # x half-lengths 96 / 48 and y lengths 96 / 192, z lengths 96 / 192 (radix-3 register FFTs)
          (96, 48, 8), (48, 96, 8), (8, 8, 48), (8, 8, 96),
          # rows shorter than the x half-length in the tiled step kernel (x padded beyond 2 nx):
          # 20 of 32, 40 and 44 of 48, 80 of 96
          (20, 8, 6), (40, 12, 8), (44, 10, 6), (80, 8, 4)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("term,tol", [(1, 2e-6), (2, 2e-6), (4, 2e-5), (8, 1e-7)])
def test_each_field_term_matches_oracle(ctx, shape, term, tol):
    mat, P = mixed_case(shape, seed=sum(shape))
    E = (2e7, -1e7, 3e7)
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 280.0, 30.0, E=E, P=P)
    o = oracle_sys(shape, CELL, mat, MATS, 280.0, 30.0, E=E)
    key = {1: "landau", 2: "grad", 4: "elec", 8: "ext"}[term]
    want = np.where(mat > 0, o.fields(P.astype(np.float64))[key], 0.0)   # zero on vacuum by contract
    got = g.get_field(term)
    if np.abs(want).max() == 0:
        assert np.abs(got).max() == 0
        return
    assert rel_err(got, want) <= tol
    assert np.all(got[:, mat == 0] == 0)


@pytest.mark.parametrize("shape,Mz", [((8, 8, 48), 96), ((8, 8, 96), 192), ((17, 9, 40), 81)])
def test_electrostatic_field_with_forced_z_padding_matches_oracle(ctx, shape, Mz):
    # by default z lengths 96 and 192 give way to the tuned 128 and 256; forcing the smallest
    # 2^a 3^b keeps the radix-3 z passes (and a generic 81-point one) pinned against the oracle,
    # and both paddings give the same field
    mat, P = mixed_case(shape, seed=sum(shape) + 1)
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 280.0, 30.0, P=P)
    default = g.get_field(4)
    g.set_fft_pad(0, 0, Mz)
    assert g.fft_pad()[2] == Mz
    got = g.get_field(4)
    o = oracle_sys(shape, CELL, mat, MATS, 280.0, 30.0)
    want = np.where(mat > 0, o.fields(P.astype(np.float64))["elec"], 0.0)
    assert rel_err(got, want) <= 2e-5
    assert rel_err(default, want) <= 2e-5


@pytest.mark.parametrize("shape", [(40, 12, 8), (20, 16, 12)])
def test_trajectory_with_rows_shorter_than_the_half_length(ctx, shape):
    # the tiled step kernel on rows of nx < Mx / 2 cells (mixed materials, vacuum holes, cross
    # terms): 24 steps, graph replays included, against the oracle trajectory
    mat, P = mixed_case(shape, seed=sum(shape) + 7)
    P *= 0.3
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 290.0, 40.0, E=(0.0, 1e7, 2e7), P=P)
    Mx = g.fft_pad()[0]
    assert shape[0] < Mx // 2
    o = oracle_sys(shape, CELL, mat, MATS, 290.0, 40.0, E=(0.0, 1e7, 2e7))
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    g.step(8, dt)
    g.energy()
    g.step(16, dt)
    want = o.run(P.astype(np.float64), dt, 24)
    assert np.abs(g.get_P() - want).max() / g.scales()[0] <= 1e-5


def test_electrostatic_field_of_uniform_slab(ctx):
    # closed form as well: uniform Pz film -> E_z ~ -Pz/(eps0 epsB) in the middle
    shape = (64, 64, 2)
    mat = np.ones((2, 64, 64), np.uint8)
    P = np.zeros((3, 2, 64, 64), np.float32); P[2] = 0.25
    g = gpu_sim(ctx, shape, (1e-9,) * 3, mat, {1: synth.BTO}, 300.0, 45.0, P=P)
    o = oracle_sys(shape, (1e-9,) * 3, mat, {1: synth.BTO}, 300.0, 45.0)
    got = g.get_field(4)
    assert rel_err(got, o.fields(P.astype(np.float64))["elec"]) <= 2e-5
    assert got[2, :, 32, 32].mean() == pytest.approx(-0.25 / (synth.EPS0 * 45.0), rel=0.05)


@pytest.mark.parametrize("shape", [(3, 5, 7), (16, 8, 6)])
def test_energy_terms_match_oracle(ctx, shape):
    mat, P = mixed_case(shape, seed=7)
    E = (1e7, 2e7, -3e7)
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, E=E, P=P)
    o = oracle_sys(shape, CELL, mat, MATS, 300.0, 45.0, E=E)
    eg, eo = g.energy(), o.energy(P.astype(np.float64))
    scale = sum(abs(eo[k]) for k in ("land", "grad", "elec", "ext"))
    for k in ("land", "grad", "elec", "ext", "total"):
        assert abs(eg[k] - eo[k]) <= 1e-6 * scale, k


def _config1():
    c = synth.CONFIG1
    shape = c["shape"]
    nx, ny, nz = shape
    mat = np.ones((nz, ny, nx), np.uint8)
    P = synth.uniform_P(shape, c["amp"], c["seed"])
    dt = c["dt_star"] / abs(coefficients(c["material"], c["T"])["a1x"])
    return c, shape, mat, P, dt


def test_config1_trajectory_parity_100_and_200_steps(ctx):
    c, shape, mat, P, dt = _config1()
    mats = {1: c["material"]}
    g = gpu_sim(ctx, shape, c["cell"], mat, mats, c["T"], c["eps_b"], P=P)
    o = oracle_sys(shape, c["cell"], mat, mats, c["T"], c["eps_b"])
    P0 = g.scales()[0]
    Po = P.astype(np.float64)
    for _ in range(2):
        g.step(100, dt)
        Po = o.run(Po, dt, 100)
        Pg = g.get_P()
        assert np.abs(Pg - Po).max() / P0 <= 1e-5
    eg, eo = g.energy(), o.energy(Po)
    scale = sum(abs(eo[k]) for k in ("land", "grad", "elec", "ext"))
    assert abs(eg["total"] - eo["total"]) <= 1e-6 * scale


def test_mixed_materials_trajectory_parity(ctx):
    shape = (12, 10, 8)
    mat, P = mixed_case(shape, seed=3)
    P *= 0.2
    E = (0.0, 0.0, 5e7)
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, E=E, P=P)
    o = oracle_sys(shape, CELL, mat, MATS, 300.0, 45.0, E=E)
    dt = 0.003 / abs(coefficients(synth.PTO, 300.0)["a1x"])
    g.step(50, dt)
    Po = o.run(P.astype(np.float64), dt, 50)
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-5


# ---- full-size workloads: sampled cells, oracle one cell at a time -----------------------------
def _oracle_field_at(shape, cell, mat, mats, T, eps_b, P, octant, cells):
    """Total field at selected cells: local terms on a 5x5x5 block, E_el by the direct sum."""
    from oracle import System, TERM_GRAD, TERM_LANDAU
    nx, ny, nz = shape
    kappa = 1.0 / (synth.EPS0 * eps_b)
    Pd = P.astype(np.float64)
    out = []
    for (x, y, z) in cells:
        x0, x1 = max(0, x - 2), min(nx, x + 3)
        y0, y1 = max(0, y - 2), min(ny, y + 3)
        z0, z1 = max(0, z - 2), min(nz, z + 3)
        sub = System((x1 - x0, y1 - y0, z1 - z0), cell, mat[z0:z1, y0:y1, x0:x1], mats, T,
                     terms=TERM_LANDAU | TERM_GRAD)
        h = sub.fields(Pd[:, z0:z1, y0:y1, x0:x1])["total"][:, z - z0, y - y0, x - x0].copy()
        dz = np.abs(z - np.arange(nz))[:, None, None]
        dy = np.abs(y - np.arange(ny))[None, :, None]
        dx = np.abs(x - np.arange(nx))[None, None, :]
        sx = np.sign(x - np.arange(nx))[None, None, :]
        sy = np.sign(y - np.arange(ny))[None, :, None]
        sz = np.sign(z - np.arange(nz))[:, None, None]
        N = [octant[c][dz, dy, dx] for c in range(6)]
        Nxy, Nxz, Nyz = N[3] * sx * sy, N[4] * sx * sz, N[5] * sy * sz
        E = np.array([np.sum(N[0] * Pd[0] + Nxy * Pd[1] + Nxz * Pd[2]),
                      np.sum(Nxy * Pd[0] + N[1] * Pd[1] + Nyz * Pd[2]),
                      np.sum(Nxz * Pd[0] + Nyz * Pd[1] + N[2] * Pd[2])])
        if mat[z, y, x]:
            h += -kappa * E
        out.append(h)
    return np.array(out)


def _sample_cells(shape, n, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    corners = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, nz // 2), (nx // 2, 0, 0), (nx - 1, ny // 2, nz - 1)]
    rand = [tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz))) for _ in range(n)]
    return corners + rand


@pytest.mark.parametrize("workload", ["bto_cube_128", "pto_sto_bilayer_256x256x64", "bto_cube_48", "bto_cube_64",
                                      "bto_cube_96", "bto_cube_96_z192"])
def test_full_size_field_and_step_at_sampled_cells(ctx, workload):
    z192 = workload.endswith("_z192")     # the 96^3 cube with its z axis padded to 192, not 256
    workload = workload.replace("_z192", "")
    if workload.startswith("bto_cube"):
        c = synth.CONFIG2
        L = int(workload.rsplit("_", 1)[1])
        shape = (L, L, L)
        nx, ny, nz = shape
        mat = np.ones((nz, ny, nx), np.uint8)
        mats = {1: c["material"]}
        T, eps_b = 300.0, c["eps_b"]
        P = synth.uniform_P(shape, c["amp"], c["seed"])
        a1 = abs(coefficients(c["material"], T)["a1x"])
    else:
        c = synth.CONFIG4
        shape = c["shape"]
        mat = synth.layer_map(shape, c["layers"])
        mats = {1: synth.PTO, 2: synth.STO}
        T, eps_b = c["T"], c["eps_b"]
        P = synth.cylinder_start(shape, c["radius"], 0.7, c["amp"], c["seed"], z_range=(32, 64))
        a1 = abs(coefficients(synth.PTO, T)["a1x"])
    cell = c["cell"]
    E = (0.0, 0.0, 1e8)
    g = gpu_sim(ctx, shape, cell, mat, mats, T, eps_b, E=E, P=P)
    if z192:
        g.set_fft_pad(0, 0, 192)
    octant = otensor.octant(shape, cell)
    cells = _sample_cells(shape, 20, 5)
    h_o = _oracle_field_at(shape, cell, mat, mats, T, eps_b, P, octant, cells) + np.array(E)[None, :]
    h_g = g.get_field(15)
    got = np.array([h_g[:, z, y, x] for (x, y, z) in cells])
    assert rel_err(got, h_o) <= 3e-5
    dt = 0.004 / a1
    g.step(1, dt)
    Pn = g.get_P()
    want = np.array([P[:, z, y, x].astype(np.float64) + dt * h_o[i] for i, (x, y, z) in enumerate(cells)])
    gotp = np.array([Pn[:, z, y, x] for (x, y, z) in cells])
    dP = np.abs(want - np.array([P[:, z, y, x] for (x, y, z) in cells])).max()
    assert np.abs(gotp - want).max() <= 3e-5 * dP + 1e-7 * g.scales()[0]


@pytest.mark.parametrize("shape", [(32, 32, 8), (24, 12, 20), (16, 16, 16)])
def test_steps_interleaved_with_energy_and_field_reads(ctx, shape):
    # energy() and get_field() leave the field spectrum in place; the next step must reuse it
    # and chunks of any length (graph replays included) must follow the oracle trajectory
    nx, ny, nz = shape
    mat = np.ones((nz, ny, nx), np.uint8)
    P = synth.uniform_P(shape, 0.05, 21)
    g = gpu_sim(ctx, shape, (1e-9,) * 3, mat, {1: synth.BTO}, 300.0, 45.0, P=P)
    o = oracle_sys(shape, (1e-9,) * 3, mat, {1: synth.BTO}, 300.0, 45.0)
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    Po = P.astype(np.float64)
    for n, probe in [(8, "energy"), (5, "field"), (16, "energy"), (1, "energy"), (2, None), (16, None)]:
        g.step(n, dt)
        Po = o.run(Po, dt, n)
        if probe == "energy":
            g.energy()
        elif probe == "field":
            g.get_field(15)
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-5


def test_ac_applied_field_trajectory(ctx):
    # E_ext(t) = E + A sin(2 pi f t + phase), sampled at each step's time, vs the oracle
    shape = (16, 12, 8)
    mat, P = mixed_case(shape, seed=9)
    P *= 0.3
    E, A, f, ph = (0.0, 0.0, 2e7), (5e7, 0.0, 1.5e8), 3.0e8, 0.4
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, E=E, P=P)
    g.set_field_ac(A, f, ph)
    g.set_time(1e-9)
    o = oracle_sys(shape, CELL, mat, MATS, 300.0, 45.0, E=E)
    o.E_ac, o.freq, o.phase = np.array(A), f, ph
    Po = P.astype(np.float64)
    t = 1e-9
    for n in (7, 16, 9):
        g.step(n, dt)
        Po = o.run(Po, dt, n, t0=t)
        t += n * dt
    assert g.time() == pytest.approx(t, rel=1e-12)
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-5
    eg, eo = g.energy(), o.energy(Po, t)
    assert abs(eg["ext"] - eo["ext"]) <= 1e-6 * sum(abs(eo[k]) for k in ("land", "grad", "elec", "ext"))


@pytest.mark.parametrize("ac", [False, True])
def test_heun_trajectory_matches_oracle(ctx, ac):
    from paper_2605_28800_b300 import tdgl
    shape = (16, 12, 8)
    mat, P = mixed_case(shape, seed=13)
    P *= 0.3
    E, A, f, ph = (0.0, 0.0, 2e7), (0.0, 4e7, 1e8), 3.0e8, 0.2
    dt = 0.006 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, E=E, P=P)
    g.set_integrator(tdgl.HEUN)
    o = oracle_sys(shape, CELL, mat, MATS, 300.0, 45.0, E=E)
    if ac:
        g.set_field_ac(A, f, ph)
        o.E_ac, o.freq, o.phase = np.array(A), f, ph
    Po = P.astype(np.float64)
    t = 0.0
    for n in (5, 16, 1):
        g.step(n, dt)
        g.energy()
        Po = o.run(Po, dt, n, t0=t, method="heun")
        t += n * dt
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-5


def test_heun_batch_equals_single(ctx):
    from paper_2605_28800_b300 import tdgl
    sims = []
    for rep in range(2):
        row = []
        for i, sh in enumerate([(16, 16, 8), (12, 10, 6)]):
            mat, P = mixed_case(sh, seed=30 + i)
            s = gpu_sim(ctx, sh, CELL, mat, MATS, 280.0, 45.0, P=P * 0.3)
            s.set_integrator(tdgl.HEUN)
            row.append(s)
        sims.append(row)
    dt = 0.004 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    for s in sims[0]:
        s.step(16, dt)
        s.step(3, dt)
    B = tdgl.Batch(ctx, sims[1])
    B.step(16, dt)
    B.step(3, dt)
    for a, b in zip(*sims):
        assert np.array_equal(a.get_P(), b.get_P())
    B.close()


@pytest.mark.parametrize("method", ["rk45", "ab3m2"])
@pytest.mark.parametrize("ac", [False, True])
def test_multistage_trajectory_matches_oracle(ctx, method, ac):
    # fixed-step RK45 (the fourth-order solution advances) and the AB3M2 PECE pair, with the
    # stage times of a time-dependent applied field, on two materials with vacuum holes
    from paper_2605_28800_b300 import tdgl
    shape = (16, 12, 8)
    mat, P = mixed_case(shape, seed=17)
    P *= 0.3
    E, A, f, ph = (0.0, 0.0, 2e7), (0.0, 4e7, 1e8), 3.0e8, 0.2
    dt = 0.01 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, E=E, P=P)
    g.set_integrator(tdgl.RK45 if method == "rk45" else tdgl.AB3M2)
    o = oracle_sys(shape, CELL, mat, MATS, 300.0, 45.0, E=E)
    if ac:
        g.set_field_ac(A, f, ph)
        o.E_ac, o.freq, o.phase = np.array(A), f, ph
    # one uninterrupted run: an energy read between calls keeps the AB3M2 history
    g.step(5, dt)
    g.energy()
    g.step(11, dt)
    Po = o.run(P.astype(np.float64), dt, 16, method=method)
    assert g.time() == pytest.approx(16 * dt, rel=1e-12)
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-5


def test_ab3m2_history_restarts_when_the_state_is_replaced(ctx):
    from paper_2605_28800_b300 import tdgl
    shape = (12, 10, 6)
    mat, P = mixed_case(shape, seed=19)
    P *= 0.3
    dt = 0.01 / abs(coefficients(synth.BTO, 300.0)["a1x"])
    g = gpu_sim(ctx, shape, CELL, mat, MATS, 290.0, 45.0, P=P)
    g.set_integrator(tdgl.AB3M2)
    g.step(6, dt)
    P1 = g.get_P()
    g.set_P(P1)                      # same state, fresh history: the next step is Heun's
    g.step(7, dt)
    o = oracle_sys(shape, CELL, mat, MATS, 290.0, 45.0)
    Po = o.run(P1.astype(np.float64), dt, 7, t0=6 * dt, method="ab3m2")
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] <= 1e-5


def test_adaptive_rk45_relaxes_to_the_same_state(ctx):
    # with a local-error tolerance well below the relax tolerance the adaptive run converges to the
    # state the fixed-step Euler relaxation reaches (near equilibrium the controller holds dt at the
    # stability edge of the stiff gradient modes, where the accepted error is at most err_tol)
    from paper_2605_28800_b300 import tdgl
    shape = (16, 16, 8)
    mat = np.ones((8, 16, 16), np.uint8)
    P = synth.uniform_P(shape, 0.01, 21)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    dt = 0.004 / a
    ref = gpu_sim(ctx, shape, CELL, mat, {1: synth.BTO}, 300.0, 45.0, P=P)
    n_euler, ok = ref.relax(dt, 1e-7, 200000, raise_on_cap=False)
    assert ok
    g = gpu_sim(ctx, shape, CELL, mat, {1: synth.BTO}, 300.0, 45.0, P=P)
    g.set_integrator(tdgl.RK45)
    g.set_adaptive(1e-8)
    n_rk, ok = g.relax(dt, 1e-7, 200000, raise_on_cap=False)
    assert ok, (n_rk, g.dt_next() / dt)
    assert g.dt_next() != dt
    e1, e2 = ref.energy(), g.energy()
    assert abs(e1["total"] - e2["total"]) <= 1e-6 * sum(abs(e1[k]) for k in ("land", "grad", "elec"))
    assert np.abs(ref.get_P() - g.get_P()).max() / g.scales()[0] < 1e-4


def test_adaptive_rk45_grows_the_step_on_a_smooth_problem_and_stays_accurate(ctx):
    # Landau only (independent cells, no stiff coupling): the controller lengthens dt several
    # times over, and the state at the time reached matches a fine fixed-step oracle run
    from paper_2605_28800_b300 import tdgl
    from oracle import TERM_LANDAU
    shape = (8, 8, 4)
    mat = np.ones((4, 8, 8), np.uint8)
    P = synth.uniform_P(shape, 0.05, 25)
    a = abs(coefficients(synth.BTO, 300.0)["a1x"])
    dt = 0.004 / a
    g = gpu_sim(ctx, shape, CELL, mat, {1: synth.BTO}, 300.0, 45.0, P=P)
    g.set_terms(tdgl.TERM_LANDAU)
    g.set_integrator(tdgl.RK45)
    g.set_adaptive(1e-6)
    g.step(30, dt)
    assert g.dt_next() > 3 * dt
    T = g.time()
    o = oracle_sys(shape, CELL, mat, {1: synth.BTO}, 300.0, 45.0, terms=TERM_LANDAU)
    n = 4000
    Po = o.run(P.astype(np.float64), T / n, n, method="rk45")
    assert np.abs(g.get_P() - Po).max() / g.scales()[0] < 1e-4


def test_multistage_integrators_are_rejected_in_batches(ctx):
    from paper_2605_28800_b300 import tdgl
    shape = (8, 8, 4)
    mat, P = mixed_case(shape, seed=23)
    a = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, P=P)
    b = gpu_sim(ctx, shape, CELL, mat, MATS, 300.0, 45.0, P=P)
    B = tdgl.Batch(ctx, [a, b])
    with pytest.raises(tdgl.TdglError):
        a.set_integrator(tdgl.RK45)
    B.close()
    a.set_integrator(tdgl.AB3M2)
    b.set_integrator(tdgl.AB3M2)
    B = tdgl.Batch(ctx, [a, b])
    with pytest.raises(tdgl.TdglError):
        B.step(2, 1e-12)
    B.close()
