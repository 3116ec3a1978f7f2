"""Parity of the post-processing kernels (current density, field lines)
with the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_1307_6720_gb300 import mhs
    return mhs


def _solved(M, pr, bz, tol=1e-13):
    import torch
    h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"],
                     M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"], pr["xi_b"], pr["xi_omega"]))
    M.mhs_set_stream(h, torch.cuda.current_stream())
    M.mhs_set_lower_bz(h, bz)
    M.mhs_solve(h, tol, M.MHS_FP64)
    return h


def _paper_pair(n=33):
    pr = S.problem(n, n, n, Lx=11.0, Ly=11.0, Lz=12.0, alpha=0.2, xi_kind=2, xi_a=0.7, xi_b=0.3,
                   xi_omega=np.pi, xi_kappa=0.1)
    sp = [S.Spot(1.0, -1.0, -1.0, 0.3), S.Spot(-1.0, 1.0, 1.0, 0.3)]
    return pr, S.spots_field(n, n, 11.0, 11.0, sp, -5.5, -5.5)


@pytest.mark.parametrize("shape", [(33, 33, 33), (17, 33, 9), (65, 17, 33)])
def test_current_density_parity(M, shape):
    nx, ny, nz = shape
    pr = S.problem(nx, ny, nz, Lx=1.0, Ly=0.8, Lz=0.9, alpha=0.4, xi_kind=1, xi_a=0.5, xi_kappa=1.0)
    bz = S.magnetogram_random(nx, ny, 1.0, 0.8, seed=9)
    h = _solved(M, pr, bz)
    phi = np.zeros((nz, ny, nx))
    M.mhs_get_phi(h, phi)
    out = [np.zeros((nz, ny, nx)) for _ in range(5)]
    M.mhs_current(h, *out)
    F = oracle.fields(pr, phi)
    want = oracle.current(pr, F["Bx"], F["By"], F["Bz"])
    for got, key in zip(out, ["jx", "jy", "jz", "jmag", "bmag"]):
        w = want[key]
        assert np.abs(got - w).max() <= 1e-11 * np.abs(w).max(), key
    M.mhs_destroy(h)


def test_field_lines_bitwise_equal_oracle_on_same_field(M):
    """With the oracle's B as input, the GPU tracer reproduces the oracle's
    lines bit for bit (both evaluate the same expressions with every FP64
    operation rounded separately), including the step at which each line
    leaves the box."""
    import torch
    pr, bz = _paper_pair(33)
    P = exact.separable_solve3d(pr, exact.separable_solve2d(pr, bz))
    F = oracle.fields(pr, P)
    rng = np.random.default_rng(17)
    seeds = np.column_stack([rng.uniform(3.0, 8.0, 200), rng.uniform(3.0, 8.0, 200), rng.uniform(0.0, 2.0, 200)])
    seeds[0] = [20.0, 1.0, 1.0]                            # outside the box
    ds, steps = 0.05, 400
    for direction in (1, -1):
        want_p, want_l = oracle.trace(pr, F["Bx"], F["By"], F["Bz"], seeds, ds, steps, direction)
        B = [torch.from_numpy(F[k]).cuda() for k in ("Bx", "By", "Bz")]
        pts = torch.zeros((len(seeds), steps + 1, 3), dtype=torch.float64, device="cuda")
        lens = torch.zeros(len(seeds), dtype=torch.int32, device="cuda")
        M.mhs_trace_field((pr["nz"], pr["ny"], pr["nx"]), (pr["Lx"], pr["Ly"], pr["Lz"]), *B,
                          torch.from_numpy(seeds).cuda(), ds, steps, direction, pts, lens,
                          torch.cuda.current_stream())
        torch.cuda.synchronize()
        got_l = lens.cpu().numpy()
        got_p = pts.cpu().numpy()
        assert np.array_equal(got_l, want_l)
        assert want_l[0] == 0 and (want_l > 1).sum() > 150 and (want_l < steps + 1).sum() > 10
        for q in range(len(seeds)):
            assert np.array_equal(got_p[q, : got_l[q]], want_p[q, : want_l[q]]), q


def test_field_lines_of_solution_host_buffers(M):
    """mhs_trace on the handle's own B with host seeds and outputs, against
    the oracle's trace of the oracle's fields of the same potential."""
    pr, bz = _paper_pair(33)
    h = _solved(M, pr, bz)
    phi = np.zeros((33, 33, 33))
    M.mhs_get_phi(h, phi)
    F = oracle.fields(pr, phi)
    rng = np.random.default_rng(23)
    seeds = np.column_stack([rng.uniform(3.0, 8.0, 40), rng.uniform(3.0, 8.0, 40), rng.uniform(0.0, 2.0, 40)])
    seeds[-1] = [-1.0, 0.0, 0.0]
    ds, steps = 0.05, 300
    got_p, got_l = M.mhs_trace(h, seeds, ds, steps)
    want_p, want_l = oracle.trace(pr, F["Bx"], F["By"], F["Bz"], seeds, ds, steps)
    assert got_l[-1] == 0 and want_l[-1] == 0
    assert (np.minimum(got_l, want_l) > 20).sum() >= 10
    for q in range(len(seeds) - 1):
        m = min(got_l[q], want_l[q])
        assert abs(int(got_l[q]) - int(want_l[q])) <= 1
        assert np.abs(got_p[q, :m] - want_p[q, :m]).max() < 1e-8
    # zero seeds and zero steps
    p0, l0 = M.mhs_trace(h, np.zeros((0, 3)), ds, steps)
    assert l0.shape == (0,)
    p1, l1 = M.mhs_trace(h, seeds[:1], ds, 0)
    assert l1[0] == 1 and np.array_equal(p1[0, 0], seeds[0])
    with pytest.raises(M.MhsError):
        M.mhs_trace(h, seeds, -0.1, 10)
    M.mhs_destroy(h)
