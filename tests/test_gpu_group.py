"""Grouped solves (mhs_group_*): many instances, one launch per multigrid
operation and level for all of them.  Each instance must come out bitwise
identical to its solo solve (same operations, same block decomposition),
whatever the mix of grids, parameters and options in the group."""
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


def _members(M, seed=0):
    """Uneven grids, xi families and options: one anisotropic (z-line) member, cycles
    ending in the separable coarse-grid solve (fast and dense transforms) or in
    the one-CTA sub-cycle."""
    specs = [
        (S.problem(33, 33, 33, alpha=0.3, xi_kind=1, xi_a=0.5, xi_kappa=1.0), {}),
        (S.problem(65, 65, 65, alpha=0.5, xi_kind=1, xi_a=0.5, xi_kappa=1.0), {}),
        (S.problem(129, 129, 65, Lz=0.5, alpha=0.4, xi_kind=2, xi_a=0.6, xi_b=0.2, xi_omega=3.0, xi_kappa=0.5), {}),
        (S.problem(17, 33, 9, Lx=0.5, Ly=1.0, Lz=0.25, alpha=0.2), {}),
        (S.problem(65, 65, 65, alpha=0.5, xi_kind=1, xi_a=0.999, xi_kappa=0.5), {}),       # z-line (auto)
        (S.problem(33, 33, 33, alpha=0.1, xi_kind=1, xi_a=0.3, xi_kappa=2.0), dict(flags=M.MHS_FLAG_NO_FMG)),
        (S.problem(65, 33, 33, Ly=0.5, Lz=0.5, alpha=0.6, xi_kind=1, xi_a=0.5, xi_kappa=1.0), dict(nu1=1, nu2=1)),
        (S.problem(65, 65, 33, Lz=0.5, alpha=0.5, xi_kind=1, xi_a=0.4, xi_kappa=1.0), dict(cut64=40, cut32=40)),
        (S.problem(5, 5, 5, alpha=0.2), {}),
        (S.problem(65, 65, 65, alpha=0.4, xi_kind=1, xi_a=0.5, xi_kappa=1.0), dict(sep_coarse=-1)),   # sub-cycle
        (S.problem(25, 25, 13, Lz=0.5, alpha=0.3, xi_kind=1, xi_a=0.4, xi_kappa=1.0), {}),   # dense transforms
    ]
    hs, prs, bzs = [], [], []
    for q, (pr, opts) in enumerate(specs):
        h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"],
                         M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"], pr["xi_b"], pr["xi_omega"]))
        if opts:
            M.mhs_set_options(h, **opts)
        bz = S.magnetogram_random(pr["nx"], pr["ny"], pr["Lx"], pr["Ly"], seed=100 * seed + q)
        M.mhs_set_lower_bz(h, bz)
        hs.append(h)
        prs.append(pr)
        bzs.append(bz)
    return hs, prs, bzs


def _phi(M, h, pr):
    out = np.zeros((pr["nz"], pr["ny"], pr["nx"]))
    M.mhs_get_phi(h, out)
    return out


ONE_PART = (1 << 64) - 1


@pytest.mark.parametrize("parts", ["default", "one", "each"])
@pytest.mark.parametrize("mode", [1, 0])
def test_group_solve_bitwise_equals_solo_solves(M, mode, parts):
    """Default partition (half the L2 per part, two launch streams), all
    instances in one part, and one part per instance on three streams."""
    hs, prs, bzs = _members(M)
    part_bytes, nstreams = {"default": (0, 0), "one": (ONE_PART, 1), "each": (1, 3)}[parts]
    g = M.mhs_group_create(hs, mode, part_bytes, nstreams)
    tol = 1e-10
    infos, sts = M.mhs_group_solve(g, len(hs), tol)
    assert all(s == M.MHS_OK for s in sts), sts
    grouped = [_phi(M, h, pr) for h, pr in zip(hs, prs)]
    for q, (h, pr) in enumerate(zip(hs, prs)):
        solo = M.mhs_solve(h, tol, mode)
        assert solo["cycles_3d"] == infos[q]["cycles_3d"] and solo["cycles_2d"] == infos[q]["cycles_2d"], q
        assert solo["rel_res_3d"] == infos[q]["rel_res_3d"], q
        assert np.array_equal(_phi(M, h, pr), grouped[q]), q
    # the anisotropic member converged in few cycles (z-line smoothing in the group)
    assert infos[4]["cycles_3d"] <= 8
    M.mhs_group_destroy(g)
    for h in hs:
        M.mhs_destroy(h)


def test_group_repeated_solves_new_bz_and_exact_solution(M):
    hs, prs, _ = _members(M)
    g = M.mhs_group_create(hs, M.MHS_MIXED)
    for rep in range(3):
        bzs = []
        for q, (h, pr) in enumerate(zip(hs, prs)):
            bz = S.magnetogram_random(pr["nx"], pr["ny"], pr["Lx"], pr["Ly"], seed=7000 + 31 * rep + q)
            M.mhs_set_lower_bz(h, bz)
            bzs.append(bz)
        infos, sts = M.mhs_group_solve(g, len(hs), 1e-11)
        assert all(s == M.MHS_OK for s in sts)
        for q in (0, 3, 8):                                 # small members against the exact discrete solution
            pr = prs[q]
            want = exact.separable_solve3d(pr, exact.separable_solve2d(pr, bzs[q]))
            got = _phi(M, hs[q], pr)
            assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want), (rep, q)
    M.mhs_group_destroy(g)
    for h in hs:
        M.mhs_destroy(h)


def test_group_per_instance_status_and_errors(M):
    hs, prs, _ = _members(M)
    M.mhs_set_options(hs[1], max_cycles=1, flags=M.MHS_FLAG_NO_FMG)
    g = M.mhs_group_create(hs, M.MHS_MIXED)
    infos, sts = M.mhs_group_solve(g, len(hs), 1e-10)
    assert sts[1] == M.MHS_ERR_NO_CONVERGENCE
    assert all(s == M.MHS_OK for q, s in enumerate(sts) if q != 1)
    M.mhs_group_destroy(g)
    with pytest.raises(M.MhsError):
        M.mhs_group_create([hs[0], hs[0]], M.MHS_MIXED)
    h_nobz = M.mhs_create(17, 17, 17, 1.0, 1.0, 1.0, 0.0, None)
    g2 = M.mhs_group_create([hs[0], h_nobz], M.MHS_FP64)
    with pytest.raises(M.MhsError) as e:
        M.mhs_group_solve(g2, 2, 1e-10)
    assert e.value.status == M.MHS_ERR_BAD_STATE
    M.mhs_group_destroy(g2)
    M.mhs_destroy(h_nobz)
    for h in hs:
        M.mhs_destroy(h)


def test_group_eager_launches_match_graph(M):
    """The host-driven form of a group solve (for profilers) runs the same
    launches as the graph: bitwise the same P and cycle counts, and as many
    launches as the graph path accounts for (per-section counts times the
    while-loop iterations)."""
    hs, prs, _ = _members(M, seed=3)
    g = M.mhs_group_create(hs, M.MHS_MIXED)
    M.mhs_group_solve(g, len(hs), 1e-10)
    n0 = M.mhs_kernel_launches()
    infos_g, _ = M.mhs_group_solve(g, len(hs), 1e-10)
    n_graph = M.mhs_kernel_launches() - n0
    ref = [_phi(M, h, pr) for h, pr in zip(hs, prs)]
    M.mhs_group_set_eager(g, True)
    n0 = M.mhs_kernel_launches()
    infos_e, sts = M.mhs_group_solve(g, len(hs), 1e-10)
    n_eager = M.mhs_kernel_launches() - n0
    assert n_graph == n_eager > 0, (n_graph, n_eager)
    assert all(s == M.MHS_OK for s in sts)
    for q, (h, pr) in enumerate(zip(hs, prs)):
        assert infos_e[q]["cycles_3d"] == infos_g[q]["cycles_3d"]
        assert np.array_equal(_phi(M, h, pr), ref[q]), q
    M.mhs_group_destroy(g)
    for h in hs:
        M.mhs_destroy(h)
