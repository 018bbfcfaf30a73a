"""The allocation-free field entry point (tdgl_elec_field_static) against tdgl_get_field and
against the FP64 oracle's electrostatic field.

tdgl_elec_field_static serves callers that cannot call cudaMalloc (hosts that own all device
memory through their own pool allocator, real-time loops that must not wait on the driver's
allocator): its scratch is one static device array.  This file is
named to be collected last, so that a run stopping at the first failure has run everything else
first; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synth
from tests.helpers import gpu_sim, mixed_case, oracle_sys

pytestmark = pytest.mark.gpu

TOL = 2e-5   # same bar as the electrostatic parity tests: relative to max|E|


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_28800_b300 import tdgl
    c = tdgl.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape,cell,with_map", [((17, 9, 5), (1e-9, 1.1e-9, 0.9e-9), True),
                                                 ((32, 32, 8), (1e-9, 1e-9, 1e-9), False),
                                                 ((1, 1, 1), (1e-9, 1e-9, 1e-9), False)])
def test_static_field_matches_get_field_on_two_calls(ctx, shape, cell, with_map):
    import torch
    from paper_2605_28800_b300 import tdgl
    nx, ny, nz = shape
    if with_map:
        mat, P = mixed_case(shape, seed=3)
    else:
        mat = np.ones((nz, ny, nx), np.uint8)
        P = synth.uniform_P(shape, 0.2, 5)
    eps_b = 45.0
    ref_sim = gpu_sim(ctx, shape, cell, mat, {1: synth.BTO, 2: synth.PTO}, 300.0, eps_b, P=P)
    ref = ref_sim.get_field(tdgl.TERM_ELEC)
    want = oracle_sys(shape, cell, mat, {1: synth.BTO, 2: synth.PTO}, 300.0, eps_b).electrostatic_field(
        P.astype(np.float64))
    want[:, mat == 0] = 0.0
    Pt = torch.from_numpy(P).cuda()
    mt = torch.from_numpy(mat).cuda() if with_map else None
    for call in range(2):
        E = torch.full_like(Pt, float("nan"))
        torch.cuda.synchronize()
        tdgl.elec_field_static(Pt, E, cell, eps_b, mat=mt)
        torch.cuda.synchronize()
        got = E.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= TOL, (call, err)
        err_o = np.abs(got - want).max() / np.abs(want).max()
        assert err_o <= TOL, (call, err_o)


def test_static_field_rejects_oversized_and_bad_arguments():
    import torch
    from paper_2605_28800_b300 import tdgl
    big = torch.zeros((3, 40, 40, 40), device="cuda")
    with pytest.raises(tdgl.TdglError) as e:
        tdgl.elec_field_static(big, torch.empty_like(big), (1e-9,) * 3, 45.0)
    assert e.value.code == tdgl.ETOOBIG
    small = torch.zeros((3, 4, 4, 4), device="cuda")
    with pytest.raises(tdgl.TdglError) as e:
        tdgl.elec_field_static(small, torch.empty_like(small), (1e-9,) * 3, -1.0)
    assert e.value.code == tdgl.EINVAL
