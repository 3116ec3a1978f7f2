"""The autotuner (mhs_autotune) times whole solves of a handle's problem and
keeps the fastest option set: it must never end slower than its start,
store the result under the problem class (found from other handles of the
class, not from other modes or classes), and the tuned solve must still
reach the exact discrete solution."""
import numpy as np
import pytest

import synthetic as S
from oracle import exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_1307_6720_gb300 import mhs
    return mhs


def _handle(M, pr, bz):
    import torch
    h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"],
                     M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"], pr["xi_b"], pr["xi_omega"]))
    M.mhs_set_stream(h, torch.cuda.current_stream())
    M.mhs_set_lower_bz(h, bz)
    return h


def test_autotune_strong_coupling_stores_class_and_solves(M):
    M.mhs_tune_clear()
    pr = S.problem(65, 65, 65, alpha=0.5, xi_kind=1, xi_a=0.999, xi_kappa=0.5)
    bz = S.magnetogram_random(65, 65, seed=41)
    h = _handle(M, pr, bz)
    assert M.mhs_tune_lookup(h, M.MHS_FP64) is None
    res = M.mhs_autotune(h, 1e-10, M.MHS_FP64, repeats=1)
    assert res["ms"] <= res["ms_start"] and res["candidates"] >= 8, res
    assert res["aniso_class"] >= 6        # 1 / (1 - xi) at the first interior plane is ~114
    # the stored class is found from another handle of the same problem class
    h2 = _handle(M, pr, S.magnetogram_random(65, 65, seed=42))
    assert M.mhs_tune_lookup(h2, M.MHS_FP64) == res["opts"]
    assert M.mhs_tune_lookup(h2, M.MHS_MIXED) is None
    # a tuned solve still reaches the exact discrete solution
    info = M.mhs_solve(h, 1e-13, M.MHS_FP64)
    phi = np.zeros((65, 65, 65))
    M.mhs_get_phi(h, phi)
    want = exact.separable_solve3d(pr, exact.separable_solve2d(pr, bz))
    assert np.linalg.norm(phi - want) < 1e-10 * np.linalg.norm(want)
    M.mhs_destroy(h)
    M.mhs_destroy(h2)


def test_autotune_isotropic_mixed_never_slower_and_clear(M):
    M.mhs_tune_clear()
    pr, bz = S.linear_mhs(65, seed=43)
    h = _handle(M, pr, bz)
    res = M.mhs_autotune(h, 1e-10, M.MHS_MIXED, repeats=2)
    assert res["ms"] <= res["ms_start"]
    assert res["aniso_class"] <= 1
    assert M.mhs_tune_lookup(h, M.MHS_MIXED) == res["opts"]
    info = M.mhs_solve(h, 1e-10, M.MHS_MIXED)
    assert info["rel_res_3d"] < 1e-10
    M.mhs_tune_clear()
    assert M.mhs_tune_lookup(h, M.MHS_MIXED) is None
    M.mhs_destroy(h)


def test_autotune_requires_bz(M):
    h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, 0.0, None)
    with pytest.raises(M.MhsError) as e:
        M.mhs_autotune(h, 1e-10, M.MHS_FP64)
    assert e.value.status == M.MHS_ERR_BAD_STATE
    M.mhs_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_tile_shapes_give_identical_solves(M, mode):
    """The thread-block shape of the red-black point passes (option tile,
    one of the autotuner's coordinates) changes how nodes are distributed
    over threads, not which values a pass computes: every shape gives the
    same P bit for bit, FP64 and mixed, including the FP32 quad passes of
    large levels (257 x 129 x 129 interior planes of 4.2 M nodes)."""
    import torch
    pr = S.problem(257, 129, 129, Lx=1.0, Ly=0.5, Lz=0.5, alpha=0.5, xi_kind=1, xi_a=0.5, xi_kappa=1.0)
    bz = S.magnetogram_random(257, 129, 1.0, 0.5, seed=43)
    h = _handle(M, pr, bz)
    P = torch.empty((129, 129, 257), dtype=torch.float64, device="cuda")
    ref = None
    for tile in range(1, 6):
        M.mhs_set_options(h, tile=tile)
        M.mhs_solve(h, 1e-10, mode)
        M.mhs_get_phi(h, P)
        got = P.cpu().numpy()
        if ref is None:
            ref = got
        assert np.array_equal(got, ref), tile
    M.mhs_destroy(h)
