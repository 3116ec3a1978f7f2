"""Allocation-free residual check (mhs_interior_residual_noalloc).

Some callers may not allocate device memory (their device memory belongs to
their own pool allocator, or they cannot afford the synchronisation a
cudaMalloc/cudaFree may cause).  For them the library offers one entry point
whose scratch lives in a fixed device array inside the library.  This test
calls it through the C ABI twice in a row, on two different problems, and
checks each result against the existing entry points: the relative residual
that mhs_solve reports and the residual the MHS_OP_RESIDUAL level hook
writes.  Solves stop early (a few cycles) so the residual is far above
rounding and the comparison can use the suite's FP64 bar of 1e-10.  A third
case gives P non-zero values on all six faces and checks the residual and
the lifted right-hand side against the oracle.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

BAR = 1e-10


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_1307_6720_gb300 import mhs
    return mhs


def _case(M, pr, bz, cycles):
    """Early-stopped FP64 solve; returns (P on the device, reported rel. residual, hook residual norm)."""
    import torch
    xi = M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"], pr["xi_b"], pr["xi_omega"])
    h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"], xi)
    M.mhs_set_options(h, max_cycles=cycles)
    M.mhs_set_lower_bz(h, bz)
    with pytest.raises(M.MhsError) as e:
        M.mhs_solve(h, 1e-12, M.MHS_FP64)
    assert e.value.status == M.MHS_ERR_NO_CONVERGENCE
    rel = e.value.info["rel_res_3d"]
    shape = (pr["nz"], pr["ny"], pr["nx"])
    P = torch.empty(shape, dtype=torch.float64, device="cuda")
    M.mhs_get_phi(h, P)
    M.mhs_level_op(h, 3, 0, M.MHS_OP_RESIDUAL, M.MHS_FP64)
    r = np.zeros(shape)
    M.mhs_level_read(h, 3, 0, M.MHS_FIELD_R, M.MHS_FP64, r)
    M.mhs_destroy(h)
    return xi, P, rel, float(np.linalg.norm(r[1:-1, 1:-1, 1:-1]))


def test_noalloc_residual_matches_solver_twice_in_a_row(M):
    import torch
    cases = [
        (S.linear_mhs(65, seed=31)[0], S.linear_mhs(65, seed=31)[1], 2),
        (S.problem(33, 17, 33, Lx=1.0, Ly=0.5, Lz=1.0, alpha=0.3, xi_kind=2, xi_a=0.7, xi_b=0.3, xi_omega=np.pi,
                   xi_kappa=0.1), S.magnetogram_random(33, 17, 1.0, 0.5, seed=32), 1),
    ]
    prepared = [_case(M, pr, bz, cyc) for pr, bz, cyc in cases]
    outs = []
    for (pr, _, _), (xi, P, rel, rnorm) in zip(cases, prepared):
        out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        M.mhs_interior_residual_noalloc(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"], xi,
                                        P, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        outs.append(o)
        assert abs(o[2] - rel) <= BAR * rel, (o, rel)
        assert abs(o[0] - rnorm) <= BAR * rnorm, (o, rnorm)
        assert abs(o[0] / o[1] - o[2]) <= 1e-15 * o[2]
    assert not np.allclose(outs[0], outs[1])


def test_noalloc_lifts_every_face_like_the_oracle(M):
    """P with Dirichlet data on all six faces: out[0] is the oracle's interior
    residual norm, out[1] the norm of the oracle's residual of P with its
    interior zeroed (the lifted right-hand side), out[2] their ratio."""
    import torch
    import oracle
    pr = S.problem(33, 17, 25, Lx=1.0, Ly=0.5, Lz=0.75, alpha=0.4, xi_kind=2, xi_a=0.6, xi_b=0.3,
                   xi_omega=np.pi, xi_kappa=0.2)
    P = np.random.default_rng(77).standard_normal((25, 17, 33))
    r = oracle.residual3d(pr, P)
    lift = P.copy()
    lift[1:-1, 1:-1, 1:-1] = 0.0
    b = oracle.residual3d(pr, lift)
    want = np.array([np.linalg.norm(r), np.linalg.norm(b), np.linalg.norm(r) / np.linalg.norm(b)])
    xi = M.xi_params(2, 0.6, 0.2, 0.3, np.pi)
    Pd = torch.from_numpy(P).cuda()
    for _ in range(2):
        out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        M.mhs_interior_residual_noalloc(33, 17, 25, 1.0, 0.5, 0.75, 0.4, xi, Pd, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.abs(o - want) <= BAR * want), (o, want)


def test_noalloc_rejects_out_of_range_inputs(M):
    import torch
    P = torch.zeros((5, 5, 5), dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MhsError) as e:
        M.mhs_interior_residual_noalloc(5, 5, 5000, 1.0, 1.0, 1.0, 0.0, None, P, out)
    assert e.value.status == M.MHS_ERR_INVALID_ARG and "limit" in str(e.value)
    with pytest.raises(M.MhsError) as e:
        M.mhs_interior_residual_noalloc(5, 5, 5, 1.0, 1.0, 1.0, 0.0, None, np.zeros((5, 5, 5)), out)
    assert e.value.status == M.MHS_ERR_INVALID_ARG
    for xi, alpha in ((M.xi_params(7, 0.5, 1.0), 0.0), (M.xi_params(1, float("nan"), 1.0), 0.0),
                      (None, float("inf"))):
        with pytest.raises(M.MhsError) as e:
            M.mhs_interior_residual_noalloc(5, 5, 5, 1.0, 1.0, 1.0, alpha, xi, P, out)
        assert e.value.status == M.MHS_ERR_INVALID_ARG
