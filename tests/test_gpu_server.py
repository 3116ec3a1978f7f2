"""Request server: continuous batching with HBM-budget admission.

Requests of several grid shapes arrive while others run; each result must be
the same as the solo solve of the same problem (bitwise: the server runs the
solo kernels), budget-limited admission must still complete every request,
and a request larger than the whole budget is rejected."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_1307_6720_gb300 import mhs
    return mhs


def _requests(n):
    out = []
    for r in range(n):
        n3 = [33, 65, 33, 17][r % 4]
        rng = S.SplitMix64(500 + r)
        alpha, a, kappa = rng.uniform(0, 0.8), rng.uniform(0, 0.95), rng.uniform(0.5, 2.0)
        out.append((n3, alpha, a, kappa, S.magnetogram_random(n3, n3, seed=500 + r)))
    return out


def _solo(M, n3, alpha, a, kappa, bz):
    h = M.mhs_create(n3, n3, n3, 1.0, 1.0, 1.0, alpha, M.xi_params(M.MHS_XI_EXP, a, kappa))
    M.mhs_set_lower_bz(h, bz)
    M.mhs_solve(h, 1e-10, M.MHS_MIXED)
    phi = np.zeros((n3, n3, n3))
    rho = np.zeros((n3, n3, n3))
    M.mhs_get_phi(h, phi)
    M.mhs_fields(h, None, None, None, None, rho)
    M.mhs_destroy(h)
    return phi, rho


@pytest.mark.parametrize("budget_mb,inflight", [(4096, 8), (60, 3)])
def test_server_results_equal_solo_solves(M, budget_mb, inflight):
    reqs = _requests(12)
    srv = M.mhs_server_create(budget_mb << 20, inflight)
    outs, tickets = [], []
    for n3, alpha, a, kappa, bz in reqs:
        phi = np.zeros((n3, n3, n3)); rho = np.zeros((n3, n3, n3))
        outs.append((phi, rho))
        tickets.append(M.mhs_server_submit(srv, n3, n3, n3, 1.0, 1.0, 1.0, alpha,
                                           M.xi_params(M.MHS_XI_EXP, a, kappa), bz, 1e-10, M.MHS_MIXED,
                                           phi=phi, rho=rho))
    results = [M.mhs_server_wait(srv, t, 120.0) for t in tickets]
    stats = M.mhs_server_stats(srv)
    M.mhs_server_destroy(srv)
    assert all(st == 0 for _, st, _ in results), results
    assert stats["completed"] == len(reqs) and stats["rejected"] == 0
    assert stats["device_bytes"] <= budget_mb << 20
    for (n3, alpha, a, kappa, bz), (phi, rho), (info, _, lat) in zip(reqs, outs, results):
        sphi, srho = _solo(M, n3, alpha, a, kappa, bz)
        assert np.array_equal(phi, sphi) and np.array_equal(rho, srho)
        assert info["rel_res_3d"] < 1e-10 and lat > 0


def test_server_rejects_request_over_budget(M):
    srv = M.mhs_server_create(1 << 20, 2)
    bz = S.magnetogram_random(65, 65, seed=1)
    t = M.mhs_server_submit(srv, 65, 65, 65, 1.0, 1.0, 1.0, 0.5, M.xi_params(M.MHS_XI_EXP, 0.5, 1.0), bz)
    info, st, lat = M.mhs_server_wait(srv, t, 60.0)
    assert st == M.MHS_ERR_REJECTED
    assert M.mhs_server_stats(srv)["rejected"] == 1
    M.mhs_server_destroy(srv)


def test_server_rejects_nonfinite_input(M):
    srv = M.mhs_server_create(1 << 30, 2)
    bz = S.magnetogram_random(17, 17, seed=1)
    bz[3, 4] = np.inf
    with pytest.raises(M.MhsError) as e:
        M.mhs_server_submit(srv, 17, 17, 17, 1.0, 1.0, 1.0, 0.5, None, bz)
    assert e.value.status == M.MHS_ERR_NONFINITE
    M.mhs_server_destroy(srv)
