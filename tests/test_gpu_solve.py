"""Whole-solve parity of the GPU path (C ABI) with the CPU oracle.

The oracle side is the exact discrete solution (separable sine transform +
tridiagonal solves, itself pinned against the multigrid oracle and a sparse
direct solve) followed by the oracle's field recovery.  Comparisons are
relative L2 norms over all nodes: 1e-10 in FP64 mode (solve run to a 1e-13
relative residual so that the solve error is far below the bar), 1e-8 in
mixed mode at the 1e-10 residual tolerance the benchmark uses.
"""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _xi(M, pr):
    return M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"], pr["xi_b"], pr["xi_omega"])


def _gpu_solve(M, pr, bz, tol, mode, device=True, opts=None):
    import torch
    h = M.mhs_create(pr["nx"], pr["ny"], pr["nz"], pr["Lx"], pr["Ly"], pr["Lz"], pr["alpha"], _xi(M, pr))
    M.mhs_set_stream(h, torch.cuda.current_stream())
    if opts:
        M.mhs_set_options(h, **opts)
    src = torch.from_numpy(bz).cuda() if device else np.ascontiguousarray(bz)
    M.mhs_set_lower_bz(h, src)
    info = M.mhs_solve(h, tol, mode)
    shape = (pr["nz"], pr["ny"], pr["nx"])
    if device:
        outs = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(6)]
        M.mhs_get_phi(h, outs[0])
        M.mhs_fields(h, *outs[1:])
        torch.cuda.synchronize()
        outs = [o.cpu().numpy() for o in outs]
    else:
        outs = [np.zeros(shape) for _ in range(6)]
        M.mhs_get_phi(h, outs[0])
        M.mhs_fields(h, *outs[1:])
    M.mhs_destroy(h)
    return info, dict(zip(["phi", "Bx", "By", "Bz", "p", "rho"], outs))


def _oracle(pr, bz):
    P = exact.exact_solution(pr, bz)
    F = oracle.fields(pr, P)
    prof = oracle.profiles(pr)
    F["phi"] = P
    F["dp"] = F["p"] - prof["pb"][:, None, None]
    F["drho"] = F["rho"] - prof["rhob"][:, None, None]
    return F


def _compare(got, want, bar):
    prof_free = dict(got)
    errs = {k: rel(got[k], want[k]) for k in ["phi", "Bx", "By", "Bz", "p", "rho"]}
    # the magnetic parts of p and rho on their own (p_b, rho_b dominate p, rho)
    nz = got["p"].shape[0]
    dp_g = got["p"] - (want["p"] - want["dp"])
    dr_g = got["rho"] - (want["rho"] - want["drho"])
    if np.linalg.norm(want["dp"]) > 0:
        errs["p-p_b"] = rel(dp_g, want["dp"])
        errs["rho-rho_b"] = rel(dr_g, want["drho"])
    bad = {k: v for k, v in errs.items() if not v < bar}
    assert not bad, (bad, errs)
    return errs


def test_potential_field_33_fp64(M):
    pr, bz = S.potential_field_33()
    info, got = _gpu_solve(M, pr, bz, 1e-13, M.MHS_FP64)
    assert info["rel_res_3d"] < 1e-13 and info["rel_res_2d"] < 1e-13
    _compare(got, _oracle(pr, bz), 1e-10)
    # odd symmetry of the +/- pair survives on the GPU
    P = got["phi"]
    assert np.abs(P + P[:, :, ::-1]).max() < 1e-11 * np.abs(P).max()


def test_linear_mhs_129_fp64(M):
    pr, bz = S.linear_mhs(129)
    info, got = _gpu_solve(M, pr, bz, 1e-13, M.MHS_FP64)
    assert info["rel_res_3d"] < 1e-13
    assert info["conv_factor"] < 0.15
    _compare(got, _oracle(pr, bz), 1e-10)


def test_linear_mhs_129_mixed(M):
    pr, bz = S.linear_mhs(129)
    info, got = _gpu_solve(M, pr, bz, 1e-10, M.MHS_MIXED)
    assert info["rel_res_3d"] < 1e-10 and info["rel_res_2d"] < 1e-10
    _compare(got, _oracle(pr, bz), 1e-8)


def test_linear_mhs_129_fp64_at_benchmark_tolerance(M):
    """At the benchmark's 1e-10 relative residual the solution error stays
    below 1e-8 (relative L2) in FP64 mode as well."""
    pr, bz = S.linear_mhs(129)
    info, got = _gpu_solve(M, pr, bz, 1e-10, M.MHS_FP64)
    assert info["rel_res_3d"] < 1e-10
    _compare(got, _oracle(pr, bz), 1e-8)


@pytest.mark.parametrize("mode", [0, 1])
def test_non_cubic_grid(M, mode):
    """129 x 129 x 65 nodes on [0,1]^2 x [0,0.5] (isotropic spacing)."""
    pr, bz = S.linear_mhs(129, seed=21, nz=65, Lz=0.5)
    info, got = _gpu_solve(M, pr, bz, 1e-13 if mode == 0 else 1e-10, mode)
    _compare(got, _oracle(pr, bz), 1e-10 if mode == 0 else 1e-8)


def test_paper_xi2_profile_anisotropic_spacing(M):
    """xi_2 family of Sect. 3.2 on 33 x 17 x 33 nodes of [0,1] x [0,0.75] x [0,1.2]."""
    pr = S.problem(33, 17, 33, Lx=1.0, Ly=0.75, Lz=1.2, alpha=0.3, xi_kind=2, xi_a=0.7, xi_b=0.3,
                   xi_omega=np.pi, xi_kappa=0.1)
    bz = S.magnetogram_random(33, 17, 1.0, 0.75, seed=4)
    info, got = _gpu_solve(M, pr, bz, 1e-13, M.MHS_FP64, opts=dict(max_cycles=400))
    _compare(got, _oracle(pr, bz), 1e-10)


def test_smallest_grid(M):
    pr = S.problem(5, 5, 5, alpha=0.5, xi_kind=1, xi_a=0.5, xi_kappa=1.0)
    bz = S.magnetogram_random(5, 5, seed=1)
    info, got = _gpu_solve(M, pr, bz, 1e-13, M.MHS_FP64)
    _compare(got, _oracle(pr, bz), 1e-10)


def test_host_and_device_buffers_agree(M):
    pr, bz = S.linear_mhs(33, seed=5)
    _, a = _gpu_solve(M, pr, bz, 1e-12, M.MHS_FP64, device=True)
    _, b = _gpu_solve(M, pr, bz, 1e-12, M.MHS_FP64, device=False)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_repeat_solves_are_bitwise_identical(M):
    pr, bz = S.linear_mhs(65, seed=6)
    _, a = _gpu_solve(M, pr, bz, 1e-10, M.MHS_MIXED)
    _, b = _gpu_solve(M, pr, bz, 1e-10, M.MHS_MIXED)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_zero_field_gives_zero_potential(M):
    pr = S.problem(17, 17, 17, alpha=0.5, xi_kind=1, xi_a=0.5, xi_kappa=1.0)
    info, got = _gpu_solve(M, pr, np.zeros((17, 17)), 1e-10, M.MHS_FP64)
    assert info["cycles_2d"] == 0 and info["cycles_3d"] == 0
    assert not np.any(got["phi"])


def test_error_paths(M):
    import torch
    h = M.mhs_create(17, 17, 17, 1.0, 1.0, 1.0, 0.5)
    with pytest.raises(M.MhsError) as e:
        M.mhs_solve(h, 1e-10)
    assert e.value.status == M.MHS_ERR_BAD_STATE
    with pytest.raises(M.MhsError) as e:
        M.mhs_fields(h, np.zeros((17, 17, 17)))
    assert e.value.status == M.MHS_ERR_BAD_STATE
    bz = S.magnetogram_random(17, 17, seed=2)
    bad = bz.copy(); bad[5, 7] = np.nan
    with pytest.raises(M.MhsError) as e:
        M.mhs_set_lower_bz(h, bad)
    assert e.value.status == M.MHS_ERR_NONFINITE
    with pytest.raises(M.MhsError) as e:
        M.mhs_solve(h, 1e-10)
    assert e.value.status == M.MHS_ERR_BAD_STATE
    M.mhs_set_lower_bz(h, bz)
    with pytest.raises(M.MhsError) as e:
        M.mhs_solve(h, 0.0)
    assert e.value.status == M.MHS_ERR_INVALID_ARG
    # forced non-convergence: one cycle cannot reach 1e-12; P stays usable
    M.mhs_set_options(h, max_cycles=1)
    with pytest.raises(M.MhsError) as e:
        M.mhs_solve(h, 1e-12)
    assert e.value.status == M.MHS_ERR_NO_CONVERGENCE
    phi = np.zeros((17, 17, 17))
    M.mhs_get_phi(h, phi)
    assert np.all(np.isfinite(phi)) and np.any(phi)
    # the handle recovers: defaults again, then a warm start needs no cycle
    M.mhs_set_options(h)
    info = M.mhs_solve(h, 1e-12)
    M.mhs_set_options(h, flags=M.MHS_FLAG_WARM)
    info2 = M.mhs_solve(h, 1e-10)
    assert info2["cycles_3d"] == 0
    M.mhs_destroy(h)


def test_set_params_matches_fresh_handle(M):
    pr, bz = S.linear_mhs(33, seed=8, alpha=0.3, a=0.8, kappa=2.0)
    h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, 0.0)
    M.mhs_set_params(h, pr["alpha"], _xi(M, pr))
    M.mhs_set_lower_bz(h, bz)
    M.mhs_solve(h, 1e-12)
    phi = np.zeros((33, 33, 33))
    M.mhs_get_phi(h, phi)
    M.mhs_destroy(h)
    _, got = _gpu_solve(M, pr, bz, 1e-12, M.MHS_FP64)
    assert np.array_equal(phi, got["phi"])


def test_mimetic_bz_divergence_free(M):
    pr, bz = S.linear_mhs(33, seed=9)
    _, got = _gpu_solve(M, pr, bz, 1e-12, M.MHS_FP64, opts=dict(flags=M.MHS_FLAG_BZ_MIMETIC))
    h = 1.0 / 32
    div = (np.gradient(got["Bx"], h, axis=2, edge_order=2) + np.gradient(got["By"], h, axis=1, edge_order=2)
           + np.gradient(got["Bz"], h, axis=0, edge_order=2))
    assert np.abs(div).max() < 1e-9 * np.abs(got["Bz"]).max() / h
    want = oracle.fields(pr, exact.exact_solution(pr, bz), bz_mode=1)
    assert rel(got["Bz"], want["Bz"]) < 1e-10


@pytest.mark.parametrize("mode", [0, 1])
def test_graph_and_eager_paths_agree_bitwise(M, mode):
    """The captured solve (conditional while nodes, device-side convergence
    test) and the eager launch sequence run the same kernels in the same
    order: identical results, cycle counts and residuals, and the launch
    count the graph path reports from its per-section counts and the number
    of while-body iterations equals the eager path's count of its launches."""
    pr, bz = S.linear_mhs(65, seed=12)
    out = []
    for timing in (False, True):   # kernel timing forces the eager path
        h = M.mhs_create(65, 65, 65, 1.0, 1.0, 1.0, pr["alpha"], _xi(M, pr))
        M.mhs_set_kernel_timing(h, timing)
        M.mhs_set_lower_bz(h, bz)
        M.mhs_solve(h, 1e-10, mode)   # first solve: capture, coefficients
        n0 = M.mhs_kernel_launches()
        info = M.mhs_solve(h, 1e-10, mode)
        n = M.mhs_kernel_launches() - n0
        phi = np.zeros((65, 65, 65))
        M.mhs_get_phi(h, phi)
        M.mhs_destroy(h)
        out.append((info, phi, n))
    (ia, pa, na), (ib, pb, nb) = out
    assert np.array_equal(pa, pb)
    for k in ("cycles_2d", "cycles_3d", "rel_res_2d", "rel_res_3d"):
        assert ia[k] == ib[k], k
    assert na == nb > 0, (na, nb)


def test_repeated_graph_launches_and_option_changes(M):
    pr, bz = S.linear_mhs(33, seed=13)
    h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, pr["alpha"], _xi(M, pr))
    M.mhs_set_lower_bz(h, bz)
    a = M.mhs_solve(h, 1e-10)
    b = M.mhs_solve(h, 1e-10)
    assert a["cycles_3d"] == b["cycles_3d"] and a["rel_res_3d"] == b["rel_res_3d"]
    M.mhs_set_options(h, nu1=1, nu2=1)           # re-captured with other sweep counts
    c = M.mhs_solve(h, 1e-10)
    assert c["cycles_3d"] > a["cycles_3d"] and c["rel_res_3d"] < 1e-10
    e = M.mhs_solve(h, 1e-6)                      # tolerance lives in device memory, not in the graph
    assert e["cycles_3d"] < c["cycles_3d"]
    M.mhs_destroy(h)


def test_batch_solve_matches_solo_solves(M):
    """Instances of different sizes and parameters solved together give
    bitwise the results of solving each alone."""
    import torch
    specs = [(33, 33, 33, 1.0, 0.2, 0.9, 0.7, 41), (65, 65, 65, 1.0, 0.6, 0.5, 1.5, 42),
             (33, 33, 17, 0.5, 0.0, 0.0, 1.0, 43), (65, 65, 33, 0.5, 0.8, 0.99, 0.5, 44)]
    solo, hs = [], []
    for nx, ny, nz, Lz, alpha, a, kappa, seed in specs:
        bz = S.magnetogram_random(nx, ny, seed=seed)
        xi = M.xi_params(M.MHS_XI_EXP, a, kappa)
        h = M.mhs_create(nx, ny, nz, 1.0, 1.0, Lz, alpha, xi)
        M.mhs_set_lower_bz(h, bz)
        info = M.mhs_solve(h, 1e-10, M.MHS_MIXED)
        phi = np.zeros((nz, ny, nx)); M.mhs_get_phi(h, phi)
        solo.append((info, phi))
        M.mhs_set_lower_bz(h, bz)
        hs.append(h)
    infos, sts = M.mhs_batch_solve(hs, 1e-10, M.MHS_MIXED)
    assert all(s == 0 for s in sts)
    for h, (info, phi), bi in zip(hs, solo, infos):
        got = np.zeros_like(phi); M.mhs_get_phi(h, got)
        assert np.array_equal(got, phi)
        assert bi["cycles_3d"] == info["cycles_3d"] and bi["rel_res_3d"] == info["rel_res_3d"]
        M.mhs_destroy(h)


def test_no_graph_flag_matches_graph(M):
    pr, bz = S.linear_mhs(33, seed=14)
    out = []
    for flags in (0, M.MHS_FLAG_NO_GRAPH):
        h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, pr["alpha"], _xi(M, pr))
        M.mhs_set_options(h, flags=flags)
        M.mhs_set_lower_bz(h, bz)
        M.mhs_solve(h, 1e-10, M.MHS_MIXED)
        phi = np.zeros((33, 33, 33)); M.mhs_get_phi(h, phi)
        M.mhs_destroy(h)
        out.append(phi)
    assert np.array_equal(out[0], out[1])


def test_mixed_mode_reaches_fp64_class_residual(M):
    """The outer residual of mixed mode is evaluated in double-float
    arithmetic (pairs of FP32 words), so defect correction with FP32 V-cycles
    drives the relative residual far below FP32 rounding, to 1e-12, and the
    result then matches the exact discrete solution like FP64 mode does."""
    pr, bz = S.linear_mhs(65, seed=15)
    info, got = _gpu_solve(M, pr, bz, 1e-12, M.MHS_MIXED)
    assert info["rel_res_3d"] < 1e-12 and info["rel_res_2d"] < 1e-12
    _compare(got, _oracle(pr, bz), 2e-10)


def test_lower_boundary_fp64_flag_in_mixed_mode(M):
    """MHS_FLAG_LOWER_FP64: the lower-boundary problem of a mixed-mode solve
    runs the FP64 cycles of FP64 mode (same cycle count and residual, bit for
    bit), the interior problem keeps the mixed loop, the solution matches the
    exact discrete one, the eager path gives the same bits as the graph, and
    groups refuse the flag in mixed mode."""
    pr, bz = S.linear_mhs(129, seed=31)
    flag = M.MHS_FLAG_LOWER_FP64
    info64, _ = _gpu_solve(M, pr, bz, 1e-12, M.MHS_FP64)
    info, got = _gpu_solve(M, pr, bz, 1e-12, M.MHS_MIXED, opts=dict(flags=flag))
    assert info["cycles_2d"] == info64["cycles_2d"] and info["rel_res_2d"] == info64["rel_res_2d"]
    assert info["rel_res_3d"] < 1e-12
    _compare(got, _oracle(pr, bz), 1e-9)
    info_e, got_e = _gpu_solve(M, pr, bz, 1e-12, M.MHS_MIXED, opts=dict(flags=flag | M.MHS_FLAG_NO_GRAPH))
    assert info_e["cycles_3d"] == info["cycles_3d"]
    for k in got:
        assert np.array_equal(got_e[k], got[k]), k
    pr2 = S.problem(17, 17, 17, alpha=0.3, xi_kind=1, xi_a=0.5, xi_kappa=1.0)
    h = M.mhs_create(17, 17, 17, 1.0, 1.0, 1.0, 0.3, _xi(M, pr2))
    M.mhs_set_options(h, flags=flag)
    with pytest.raises(M.MhsError):
        M.mhs_group_create([h], M.MHS_MIXED)
    g = M.mhs_group_create([h], M.MHS_FP64)   # FP64 solves ignore the flag
    M.mhs_group_destroy(g)
    M.mhs_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_full_multigrid_start_saves_cycles_same_solution(M, mode):
    """The full-multigrid first cycle (default) reaches the tolerance in fewer
    cycles than plain V-cycles from P = 0, and both match the exact discrete
    solution."""
    pr, bz = S.linear_mhs(129, seed=18)
    want = _oracle(pr, bz)
    info_f, got_f = _gpu_solve(M, pr, bz, 1e-12, mode)
    info_v, got_v = _gpu_solve(M, pr, bz, 1e-12, mode, opts=dict(flags=M.MHS_FLAG_NO_FMG))
    assert info_f["cycles_3d"] < info_v["cycles_3d"], (info_f, info_v)
    assert info_f["cycles_2d"] <= info_v["cycles_2d"]
    _compare(got_f, want, 1e-9)
    _compare(got_v, want, 1e-9)


_PAPER_XI = {"xi1": dict(xi_kind=1, xi_a=0.7, xi_kappa=0.2),
             "xi2": dict(xi_kind=2, xi_a=0.7, xi_b=0.3, xi_omega=np.pi, xi_kappa=0.1)}


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("xi", ["xi1", "xi2"])
def test_paper_two_footpoint_workload(M, xi, mode):
    """The workload of Sect. 3.2: 129^3 nodes on [-5.5,5.5]^2 x [0,12] (the
    whole background atmosphere, transition region included), both xi
    families of Sect. 3.2, alpha = 0.2, two opposite footpoints of width 0.3.
    Phi, B, p and rho match the exact discrete solution.  The footpoints span
    about four nodes, so the differenced fields amplify the solve's error
    about a hundredfold over Phi: mixed mode runs to a 3e-11 residual here
    (1e-10 leaves B_z within a few per cent of the 1e-8 bar, either side)."""
    n = 129
    pr = S.problem(n, n, n, Lx=11.0, Ly=11.0, Lz=12.0, alpha=0.2, **_PAPER_XI[xi])
    sp = [S.Spot(1.0, -1.0, -1.0, 0.3), S.Spot(-1.0, 1.0, 1.0, 0.3)]
    bz = S.spots_field(n, n, 11.0, 11.0, sp, -5.5, -5.5)
    info, got = _gpu_solve(M, pr, bz, 1e-13 if mode == 0 else 3e-11, mode, opts=dict(max_cycles=200))
    _compare(got, _oracle(pr, bz), 1e-10 if mode == 0 else 1e-8)


def test_paper_three_source_force_free(M):
    """Sect. 3.1: xi = 0, alpha = 0.4, three Gaussian sources of width 0.3 on
    [-5.5,5.5]^2 x [0,12], 65^3 nodes; with xi = 0 the plasma terms vanish and
    p, rho equal the background atmosphere exactly."""
    n = 65
    pr = S.problem(n, n, n, Lx=11.0, Ly=11.0, Lz=12.0, alpha=0.4)
    bz = S.magnetogram_three_sources(n, n)
    info, got = _gpu_solve(M, pr, bz, 1e-13, M.MHS_FP64)
    want = _oracle(pr, bz)
    _compare(got, want, 1e-10)
    assert not np.any(want["dp"]) and not np.any(want["drho"])
    assert rel(got["p"], want["p"]) < 1e-13 and rel(got["rho"], want["rho"]) < 1e-13


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", [(65, 65, 65), (129, 129, 65)])
def test_zline_solve_with_strong_vertical_coupling(M, shape, mode):
    """xi(z) = 0.999 exp(-z/2): near the base the horizontal coupling nearly
    vanishes.  With z-line smoothing the solve needs few cycles (point
    red-black Gauss-Seidel needs several times more) and reaches the exact
    discrete solution.  The near-degenerate horizontal coupling raises the
    condition number, so both modes solve to a residual well below 1e-10
    before the fields are compared (mixed mode to 5e-12: its double-float
    outer residual levels off near 1e-12 on the 129 x 129 lower-boundary
    plane)."""
    nx, ny, nz = shape
    Lz = (nz - 1) / (nx - 1)
    pr = S.problem(nx, ny, nz, Lz=Lz, alpha=0.5, xi_kind=1, xi_a=0.999, xi_kappa=0.5)
    bz = S.magnetogram_random(nx, ny, seed=31)
    tol = 1e-13 if mode == 0 else 5e-12
    info_l, got = _gpu_solve(M, pr, bz, tol, mode, opts=dict(flags=M.MHS_FLAG_ZLINE))
    info_p, _ = _gpu_solve(M, pr, bz, tol, mode, opts=dict(max_cycles=400, flags=M.MHS_FLAG_POINT))
    info_a, _ = _gpu_solve(M, pr, bz, tol, mode)          # default: chosen from the anisotropy class
    assert info_a["cycles_3d"] == info_l["cycles_3d"]
    assert info_l["cycles_3d"] <= 10, info_l
    assert info_p["cycles_3d"] >= 2 * info_l["cycles_3d"], (info_p, info_l)
    _compare(got, _oracle(pr, bz), 1e-10 if mode == 0 else 1e-8)


@pytest.mark.parametrize("mode", [1, 0])
@pytest.mark.parametrize("case", ["lin129", "xi2_aniso", "paper", "strong", "small", "gemm"])
def test_separable_inner_solver_reaches_exact_solution(M, case, mode):
    """The exact separable solver (sine transforms and one tridiagonal system
    per mode) for the correction equation.  Mixed mode, in FP32: every outer
    step cuts the error by about the FP32 rounding level, so a few steps
    reach a 5e-12 residual (near the double-float floor of the 129 x 129
    lower-boundary plane).  FP64 mode: a direct FP64 solve per step (fast
    transforms only; the 49 x 97 x 25 grid falls back to V-cycles).  Fields
    match the exact discrete solution to the FP64 bar."""
    if case == "lin129":
        pr, bz = S.linear_mhs(129, seed=51)
    elif case == "xi2_aniso":
        pr = S.problem(65, 33, 17, Lx=1.0, Ly=0.75, Lz=0.3, alpha=0.3, xi_kind=2, xi_a=0.7, xi_b=0.3,
                       xi_omega=np.pi, xi_kappa=0.1)
        bz = S.magnetogram_random(65, 33, 1.0, 0.75, seed=52)
    elif case == "paper":
        pr = S.problem(129, 129, 129, Lx=11.0, Ly=11.0, Lz=12.0, alpha=0.2, **_PAPER_XI["xi2"])
        sp = [S.Spot(1.0, -1.0, -1.0, 0.3), S.Spot(-1.0, 1.0, 1.0, 0.3)]
        bz = S.spots_field(129, 129, 11.0, 11.0, sp, -5.5, -5.5)
    elif case == "strong":
        pr = S.problem(65, 65, 65, alpha=0.5, xi_kind=1, xi_a=0.999, xi_kappa=0.5)
        bz = S.magnetogram_random(65, 65, seed=53)
    elif case == "small":
        pr = S.problem(5, 9, 5, Ly=2.0, alpha=0.4)
        bz = S.magnetogram_random(5, 9, 1.0, 2.0, seed=54)
    else:   # nx - 1 = 48, ny - 1 = 96: not powers of two, the sine transforms run as matrix products
        pr = S.problem(49, 97, 25, Ly=2.0, Lz=0.5, alpha=0.4, xi_kind=1, xi_a=0.6, xi_kappa=1.0)
        bz = S.magnetogram_random(49, 97, 1.0, 2.0, seed=55)
    tol = 5e-12 if mode == 1 else 1e-13
    info, got = _gpu_solve(M, pr, bz, tol, mode, opts=dict(flags=M.MHS_FLAG_SEPARABLE))
    if mode == 1:
        assert info["cycles_3d"] <= 4 and info["cycles_2d"] <= 4, info
    elif case != "gemm":
        # FP64 direct solves: one step leaves only rounding, a second at most
        assert info["cycles_3d"] <= 3 and info["cycles_2d"] <= 3, info
    _compare(got, _oracle(pr, bz), 1e-10)


@pytest.mark.parametrize("mode", [0, 1])
def test_separable_solve_follows_parameter_changes(M, mode):
    """The separable solver's mode systems take alpha^2 from the level's
    coefficient table, so a captured solve replayed after mhs_set_params
    solves the new problem (same result as a fresh handle)."""
    pr, bz = S.linear_mhs(33, seed=61, alpha=0.6, a=0.7, kappa=1.5)
    h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, 0.1, None)
    M.mhs_set_options(h, flags=M.MHS_FLAG_SEPARABLE)
    M.mhs_set_lower_bz(h, bz)
    M.mhs_solve(h, 1e-11, mode)                  # captured with alpha = 0.1, xi = 0
    M.mhs_set_params(h, pr["alpha"], _xi(M, pr))
    M.mhs_solve(h, 1e-11, mode)
    phi = np.zeros((33, 33, 33))
    M.mhs_get_phi(h, phi)
    M.mhs_destroy(h)
    _, fresh = _gpu_solve(M, pr, bz, 1e-11, mode, opts=dict(flags=M.MHS_FLAG_SEPARABLE))
    assert np.array_equal(phi, fresh["phi"])
    assert rel(phi, exact.exact_solution(pr, bz)) < (1e-10 if mode == 0 else 1e-8)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("case", ["lin129", "nonpow2", "aniso"])
def test_exact_coarse_grid_solve(M, case, mode):
    """V-cycles whose coarse-grid system is solved exactly by the separable
    solver (the default, sep_coarse) reach the exact discrete solution like
    cycles that descend to the one-CTA sub-cycle, in no more cycles; on a grid
    of 2^k 3 + 1 nodes the coarse solve runs as dense transforms."""
    if case == "lin129":
        pr, bz = S.linear_mhs(129, seed=71)
    elif case == "nonpow2":
        pr = S.problem(97, 97, 49, Lz=0.5, alpha=0.4, xi_kind=1, xi_a=0.6, xi_kappa=1.0)
        bz = S.magnetogram_random(97, 97, seed=72)
    else:
        pr = S.problem(65, 33, 65, Ly=0.5, Lz=0.25, alpha=0.3, xi_kind=2, xi_a=0.7, xi_b=0.3,
                       xi_omega=np.pi, xi_kappa=0.1)
        bz = S.magnetogram_random(65, 33, 1.0, 0.5, seed=73)
    tol = 1e-13 if mode == 0 else 3e-11   # mixed: second differences (rho) amplify the residual ~100x
    want = _oracle(pr, bz)
    info_e, got_e = _gpu_solve(M, pr, bz, tol, mode)
    info_s, got_s = _gpu_solve(M, pr, bz, tol, mode, opts=dict(sep_coarse=-1))
    for got in (got_e, got_s):
        _compare(got, want, 1e-10 if mode == 0 else 1e-8)
    assert info_e["cycles_3d"] <= info_s["cycles_3d"], (info_e, info_s)
    assert info_e["cycles_2d"] <= info_s["cycles_2d"] + 1, (info_e, info_s)


def test_captured_solves_cached_per_option_set(M):
    """Switching options replays the solve captured for each option set:
    results for an option set are bitwise the same before and after other
    option sets ran, also once more sets ran than the cache keeps (8)."""
    pr, bz = S.linear_mhs(33, seed=81)
    h = M.mhs_create(33, 33, 33, 1.0, 1.0, 1.0, pr["alpha"], _xi(M, pr))
    M.mhs_set_lower_bz(h, bz)
    sets = [dict(), dict(nu1=1, nu2=1), dict(sep_coarse=-1), dict(cut64=40, cut32=40), dict(nu1=3, nu2=1),
            dict(flags=M.MHS_FLAG_NO_FMG), dict(sep_coarse=1000), dict(nu1=1, nu2=2), dict(nu1=2, nu2=1),
            dict(flags=M.MHS_FLAG_ZLINE)]

    def run(opts, mode):
        M.mhs_set_options(h, **opts)
        info = M.mhs_solve(h, 1e-10, mode)
        phi = np.zeros((33, 33, 33))
        M.mhs_get_phi(h, phi)
        return info, phi

    for mode in (0, 1):
        first = [run(o, mode) for o in sets]
        again = [run(o, mode) for o in reversed(sets)][::-1]
        for (ia, pa), (ib, pb), o in zip(first, again, sets):
            assert np.array_equal(pa, pb), o
            assert ia["cycles_3d"] == ib["cycles_3d"] and ia["rel_res_3d"] == ib["rel_res_3d"], o
    M.mhs_destroy(h)
