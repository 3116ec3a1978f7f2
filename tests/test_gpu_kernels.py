"""Operation-by-operation parity of the CUDA kernels with the CPU oracle,
through the C-ABI level hooks (the kernels the solver itself runs).

Grids are small, odd and non-cubic so several thread blocks and ragged
tails are exercised.  FP64 kernels agree with the oracle to a few ulp (the
GPU multiplies by a precomputed 1/d where the oracle divides by d, and sums
in a different order); FP32 kernels agree to FP32 rounding.
"""
import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

XI2 = dict(xi_kind=2, xi_a=0.7, xi_b=0.3, xi_omega=np.pi, xi_kappa=0.1)


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_1307_6720_gb300 import mhs
    return mhs


SHAPES = [(17, 9, 13), (33, 17, 9), (65, 33, 33), (5, 5, 5)]


def _make(M, nx, ny, nz, Lx=1.0, Ly=0.6, Lz=0.8, alpha=0.7, xi=XI2):
    """A handle on red-black point smoothing (the oracle's default smoother),
    whatever smoother the anisotropy of the grid would select, whose V-cycles
    descend to the coarsest level (as the oracle's do by default)."""
    pr = S.problem(nx, ny, nz, Lx=Lx, Ly=Ly, Lz=Lz, alpha=alpha, **xi)
    h = M.mhs_create(nx, ny, nz, Lx, Ly, Lz, alpha,
                     M.xi_params(xi["xi_kind"], xi["xi_a"], xi["xi_kappa"], xi.get("xi_b", 0), xi.get("xi_omega", 0)))
    M.mhs_set_options(h, flags=M.MHS_FLAG_POINT, sep_coarse=-1)
    return pr, h


def _read(M, h, dim, level, field, prec):
    nx, ny, nz = M.mhs_level_shape(h, dim, level)
    out = np.zeros((nz, ny, nx)) if dim == 3 else np.zeros((ny, nx))
    M.mhs_level_read(h, dim, level, field, prec, out)
    return out


def _tol(prec):
    return 2e-13 if prec == 0 else 3e-6


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_smooth_parity_3d(M, shape, prec):
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz)
    rng = np.random.default_rng(nx * 7 + ny)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 50
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:   # the FP32 kernels see the rounded inputs
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    for _ in range(2):
        M.mhs_level_op(h, 3, 0, M.MHS_OP_SMOOTH, prec)
    got = _read(M, h, 3, 0, M.MHS_FIELD_U, prec)
    want = oracle.rbgs3d(pr, u, f, 2)
    assert _rel(got, want) < _tol(prec) * 10
    M.mhs_destroy(h)


@pytest.mark.parametrize("shape", [(17, 17, 9), (33, 33, 17), (9, 9, 33), (67, 67, 11)])
def test_fp64_smooth_with_equal_xy_coefficients(M, shape):
    """FP64 sweeps on planes whose x and y coefficients are equal (h_x = h_y,
    as in the linear-MHS workloads): the colour passes agree with the oracle's
    red-black sweeps to rounding in 3D and on the lower-boundary level, and
    the fused out-of-place FP64 sweep gives bitwise the same iterate."""
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + nz)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 30
    out = []
    for flags in (0, M.MHS_FLAG_FUSED_SWEEP64):
        pr, h = _make(M, nx, ny, nz, Ly=1.0)
        M.mhs_set_options(h, flags=flags | M.MHS_FLAG_POINT, sep_coarse=-1)
        M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, 0, u)
        M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, 0, f)
        for _ in range(3):
            M.mhs_level_op(h, 3, 0, M.MHS_OP_SMOOTH, 0)
        out.append(_read(M, h, 3, 0, M.MHS_FIELD_U, 0))
        if flags == 0:   # the lower-boundary level: 5-point passes
            u2 = rng.standard_normal((ny, nx))
            f2 = rng.standard_normal((ny, nx)) * 30
            M.mhs_level_write(h, 2, 0, M.MHS_FIELD_U, 0, u2)
            M.mhs_level_write(h, 2, 0, M.MHS_FIELD_F, 0, f2)
            for _ in range(3):
                M.mhs_level_op(h, 2, 0, M.MHS_OP_SMOOTH, 0)
            assert _rel(_read(M, h, 2, 0, M.MHS_FIELD_U, 0), oracle.rbgs2d(pr, u2, f2, 3)) < 1e-12
        M.mhs_destroy(h)
    assert np.array_equal(out[0], out[1])
    assert _rel(out[0], oracle.rbgs3d(pr, u, f, 3)) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_residual_parity_3d(M, shape, prec):
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx))
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    M.mhs_level_op(h, 3, 0, M.MHS_OP_RESIDUAL, prec)
    got = _read(M, h, 3, 0, M.MHS_FIELD_R, prec)
    want = oracle.residual3d(pr, u, f)
    sl = (slice(1, -1),) * 3
    scale = np.abs(u).max() * 4 * (nx - 1) ** 2 / pr["Lx"] ** 2
    assert np.abs(got[sl] - want[sl]).max() < _tol(prec) * scale
    M.mhs_destroy(h)


@pytest.mark.parametrize("shape", [(33, 17, 9), (65, 33, 33), (17, 9, 13)])
def test_residual_after_sweep_vanishes_on_black_nodes(M, shape):
    """FP64 cycles compute the residual that follows a red-black sweep on red
    nodes only and store 0 on black ones.  Its premise, checked on the GPU
    path: after one sweep (red, then black) the full residual of every black
    node (i + j + k odd) is rounding, at most 1e-12 of the largest red one."""
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz)
    rng = np.random.default_rng(11)
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, 0, rng.standard_normal((nz, ny, nx)))
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, 0, rng.standard_normal((nz, ny, nx)) * 50)
    M.mhs_level_op(h, 3, 0, M.MHS_OP_SMOOTH, 0)
    M.mhs_level_op(h, 3, 0, M.MHS_OP_RESIDUAL, 0)
    r = _read(M, h, 3, 0, M.MHS_FIELD_R, 0)
    M.mhs_destroy(h)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inner = (i > 0) & (i < nx - 1) & (j > 0) & (j < ny - 1) & (k > 0) & (k < nz - 1)
    black = inner & ((i + j + k) % 2 == 1)
    red = inner & ((i + j + k) % 2 == 0)
    assert np.abs(r[red]).max() > 0
    assert np.abs(r[black]).max() <= 1e-12 * np.abs(r[red]).max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("shape", [(33, 17, 9), (67, 35, 19)])
def test_red_restriction_equals_full_restriction(M, dim, prec, shape):
    """The restriction the FP64 V-cycles apply to a residual taken right after
    a red-black sweep reads only the red nodes (i+j+k even) of the 27-point
    stencil; on a residual that is +0 at every black node it gives the values
    of the full restriction (same sums, the zero terms left out) and the
    oracle's full weighting."""
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz)
    rng = np.random.default_rng(17)
    fine = (nz, ny, nx) if dim == 3 else (ny, nx)
    r = rng.standard_normal(fine)
    idx = np.indices(fine).sum(axis=0)
    r[idx % 2 == 1] = 0.0
    inner = (slice(1, -1),) * len(fine)
    mask = np.zeros(fine, bool); mask[inner] = True
    r[~mask] = 0.0
    out = []
    for op in (M.MHS_OP_RESTRICT, M.MHS_OP_RESTRICT_RED):
        M.mhs_level_write(h, dim, 0, M.MHS_FIELD_R, prec, r)
        M.mhs_level_op(h, dim, 0, op, prec)
        out.append(_read(M, h, dim, 1, M.MHS_FIELD_F, prec))
    assert np.array_equal(out[0], out[1])
    want = oracle.restrict(r if prec == 0 else r.astype(np.float32).astype(np.float64))
    cin = (slice(1, -1),) * len(fine)
    assert _rel(out[1][cin], want[cin]) < _tol(prec)
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [3, 2])
def test_restriction_and_prolongation_parity(M, dim, prec):
    nx, ny, nz = 33, 17, 9
    pr, h = _make(M, nx, ny, nz)
    rng = np.random.default_rng(5)
    fine = (nz, ny, nx) if dim == 3 else (ny, nx)
    r = rng.standard_normal(fine)
    inner = (slice(1, -1),) * len(fine)
    mask = np.zeros(fine, bool); mask[inner] = True
    r[~mask] = 0.0
    M.mhs_level_write(h, dim, 0, M.MHS_FIELD_R, prec, r)
    M.mhs_level_op(h, dim, 0, M.MHS_OP_RESTRICT, prec)
    fc = _read(M, h, dim, 1, M.MHS_FIELD_F, prec)
    want = oracle.restrict(r if prec == 0 else r.astype(np.float32).astype(np.float64))
    cin = (slice(1, -1),) * len(fine)
    assert _rel(fc[cin], want[cin]) < _tol(prec)
    # prolongation + correction
    cs = oracle.coarse_shape(fine)
    ec = rng.standard_normal(cs)
    cm = np.zeros(cs, bool); cm[(slice(1, -1),) * len(cs)] = True
    ec[~cm] = 0.0
    uf = rng.standard_normal(fine)
    M.mhs_level_write(h, dim, 1, M.MHS_FIELD_U, prec, ec)
    M.mhs_level_write(h, dim, 0, M.MHS_FIELD_U, prec, uf)
    M.mhs_level_op(h, dim, 0, M.MHS_OP_PROLONG, prec)
    got = _read(M, h, dim, 0, M.MHS_FIELD_U, prec)
    if prec == 1:
        ec, uf = ec.astype(np.float32).astype(np.float64), uf.astype(np.float32).astype(np.float64)
    assert _rel(got, oracle.prolong_add(ec, uf)) < _tol(prec)
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_smooth_and_residual_parity_2d(M, prec):
    nx, ny = 65, 33
    pr, h = _make(M, nx, ny, 9, Lx=1.0, Ly=0.5)
    rng = np.random.default_rng(8)
    u = rng.standard_normal((ny, nx)); u[0] = u[-1] = 0; u[:, 0] = u[:, -1] = 0
    f = rng.standard_normal((ny, nx)) * 100
    M.mhs_level_write(h, 2, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, 2, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    M.mhs_level_op(h, 2, 0, M.MHS_OP_SMOOTH, prec)
    got = _read(M, h, 2, 0, M.MHS_FIELD_U, prec)
    want = oracle.rbgs2d(pr, u, f, 1)
    assert _rel(got, want) < _tol(prec) * 10
    M.mhs_level_op(h, 2, 0, M.MHS_OP_RESIDUAL, prec)
    r = _read(M, h, 2, 0, M.MHS_FIELD_R, prec)
    rw = oracle.residual2d(pr, want, f)
    scale = np.abs(want).max() * 4 * (nx - 1) ** 2
    assert np.abs(r[1:-1, 1:-1] - rw[1:-1, 1:-1]).max() < _tol(prec) * scale * 10
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [3, 2])
def test_coarse_solve_reaches_coarse_solution(M, dim, prec):
    """The one-CTA coarsest-level solve returns the solution of the coarse
    system (checked by the oracle's residual on that grid)."""
    nx, ny, nz = 65, 65, 33
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=1.0, Lz=0.5)
    L = M.mhs_num_levels(h, dim) - 1
    cshape = M.mhs_level_shape(h, dim, L)
    shape = cshape[::-1] if dim == 3 else cshape[1::-1]
    rng = np.random.default_rng(9)
    f = rng.standard_normal(shape)
    M.mhs_level_write(h, dim, L, M.MHS_FIELD_F, prec, f)
    M.mhs_level_op(h, dim, L, M.MHS_OP_COARSE, prec)
    u = _read(M, h, dim, L, M.MHS_FIELD_U, prec)
    fm = f.copy()
    fm[(0,) if dim == 2 else (0,)] = 0
    if dim == 3:
        r = oracle.residual3d(pr, u, f)
        fi = f[1:-1, 1:-1, 1:-1]
    else:
        r = oracle.residual2d(pr, u, f)
        fi = f[1:-1, 1:-1]
    assert np.linalg.norm(r) <= (1e-12 if prec == 0 else 1e-5) * np.linalg.norm(fi)
    M.mhs_destroy(h)


def _level_problem(M, h, pr, dim, level):
    nx, ny, nz = M.mhs_level_shape(h, dim, level)
    return S.problem(nx, ny, nz if dim == 3 else 3, Lx=pr["Lx"], Ly=pr["Ly"], Lz=pr["Lz"], alpha=pr["alpha"],
                     **{k: pr[k] for k in ("xi_kind", "xi_a", "xi_b", "xi_omega", "xi_kappa")})


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("shape", [(33, 17, 9), (65, 33, 33), (25, 13, 13), (49, 65, 17)])
def test_exact_op_parity(M, shape, dim, prec):
    """The separable solve of one level (sine transforms in x and y, a
    tridiagonal system per mode along z) against a sparse direct solve of the
    level's rediscretised operator, on every level it accepts: fast
    transforms (nx - 1, ny - 1 powers of two) and dense ones (short rows)."""
    from oracle import exact
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=0.6, Lz=0.8)
    rng = np.random.default_rng(nx + ny + nz + dim)
    for level in range(M.mhs_num_levels(h, dim)):
        lx, ly, lz = M.mhs_level_shape(h, dim, level)
        fast = (lx - 1) & (lx - 2) == 0 and (ly - 1) & (ly - 2) == 0
        if not (fast or (lx <= 66 and ly <= 66)):
            with pytest.raises(RuntimeError):
                M.mhs_level_op(h, dim, level, M.MHS_OP_EXACT, prec)
            continue
        prl = _level_problem(M, h, pr, dim, level)
        shape_l = (lz, ly, lx) if dim == 3 else (ly, lx)
        f = rng.standard_normal(shape_l) * 10
        if prec == 1:
            f = f.astype(np.float32).astype(np.float64)
        M.mhs_level_write(h, dim, level, M.MHS_FIELD_U, prec, np.zeros(shape_l))
        M.mhs_level_write(h, dim, level, M.MHS_FIELD_F, prec, f)
        M.mhs_level_op(h, dim, level, M.MHS_OP_EXACT, prec)
        got = _read(M, h, dim, level, M.MHS_FIELD_U, prec)
        if dim == 3:
            want = exact.kron_solve3d(prl, np.zeros((ly, lx)), f)
        else:
            want = exact.kron_solve2d(prl, -f)
        assert _rel(got, want) < (1e-12 if prec == 0 else 2e-5), (level, (lx, ly, lz))
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("shape", [(65, 33, 17), (49, 25, 37), (17, 9, 13), (5, 5, 5), (193, 97, 41)])
def test_fused_residual_restriction_equals_separate_launches(M, shape, dim, prec):
    """The residual + full-weighting restriction pass the V-cycles run
    (MHS_OP_RESID_RESTRICT: tiles of 16 x 8 coarse nodes, chunks of coarse
    planes, the fine residual kept in shared memory) equals the residual
    launch followed by the restriction launch bit for bit, on every level
    with a coarser one: ragged tiles, odd and even coarse counts, the zeroed
    coarse iterate; and the restriction of the oracle's residual within the
    kernel tolerance."""
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=(ny - 1) / (nx - 1), Lz=(nz - 1) / (nx - 1))
    rng = np.random.default_rng(nx + 3 * ny + 7 * nz + dim)
    for level in range(M.mhs_num_levels(h, dim) - 1):
        lx, ly, lz = M.mhs_level_shape(h, dim, level)
        cx, cy, cz = M.mhs_level_shape(h, dim, level + 1)
        shp = (lz, ly, lx) if dim == 3 else (ly, lx)
        cshp = (cz, cy, cx) if dim == 3 else (cy, cx)
        u, f = rng.standard_normal(shp), rng.standard_normal(shp)
        M.mhs_level_write(h, dim, level, M.MHS_FIELD_U, prec, u)
        M.mhs_level_write(h, dim, level, M.MHS_FIELD_F, prec, f)
        M.mhs_level_op(h, dim, level, M.MHS_OP_RESIDUAL, prec)
        M.mhs_level_op(h, dim, level, M.MHS_OP_RESTRICT, prec)
        want = _read(M, h, dim, level + 1, M.MHS_FIELD_F, prec)
        M.mhs_level_write(h, dim, level + 1, M.MHS_FIELD_F, prec, np.full(cshp, 7.0))
        M.mhs_level_write(h, dim, level + 1, M.MHS_FIELD_U, prec, np.full(cshp, 5.0))
        M.mhs_level_op(h, dim, level, M.MHS_OP_RESID_RESTRICT, prec)
        got = _read(M, h, dim, level + 1, M.MHS_FIELD_F, prec)
        uc = _read(M, h, dim, level + 1, M.MHS_FIELD_U, prec)
        inner = (slice(1, -1),) * (3 if dim == 3 else 2)
        assert np.array_equal(got[inner], want[inner]), (level, np.abs(got - want)[inner].max())
        assert np.all(uc[inner] == 0.0)
        prl = _level_problem(M, h, pr, dim, level)
        uu = _read(M, h, dim, level, M.MHS_FIELD_U, prec)
        ff = _read(M, h, dim, level, M.MHS_FIELD_F, prec)
        r = oracle.residual3d(prl, uu, ff) if dim == 3 else oracle.residual2d(prl, uu, ff)
        assert _rel(got[inner], oracle.restrict(r)[inner]) < _tol(prec) * 10, level
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(65, 65, 65), (129, 65, 33), (33, 17, 9), (257, 257, 17), (17, 33, 5)])
def test_plane_transforms_equal_staged_transforms_bitwise(M, shape, prec):
    """The per-plane separable solve (row and column transforms of a plane in
    one thread-block cluster, columns read from the other CTAs' shared
    memory) performs the staged solve's operations on every line: on every
    level with fast transforms, 2D and 3D, FP64 and FP32, its result equals
    the staged passes' (MHS_FLAG_STAGED_TRANSFORMS) bit for bit.  The launch
    counts show which path ran: one kernel for a lower-boundary level, three
    for an interior level (forward transforms, mode solves, inverse
    transforms), against five staged launches."""
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=(ny - 1) / (nx - 1), Lz=(nz - 1) / (nx - 1))
    rng = np.random.default_rng(nx * ny + nz)
    checked = 0
    for dim in (3, 2):
        for level in range(M.mhs_num_levels(h, dim)):
            lx, ly, lz = M.mhs_level_shape(h, dim, level)
            if not ((lx - 1) & (lx - 2) == 0 and (ly - 1) & (ly - 2) == 0):
                continue
            shape_l = (lz, ly, lx) if dim == 3 else (ly, lx)
            f = rng.standard_normal(shape_l) * 10
            outs, counts = [], []
            for flags in (0, M.MHS_FLAG_STAGED_TRANSFORMS):
                M.mhs_set_options(h, flags=flags)
                M.mhs_level_write(h, dim, level, M.MHS_FIELD_U, prec, np.zeros(shape_l))
                M.mhs_level_write(h, dim, level, M.MHS_FIELD_F, prec, f)
                M.mhs_level_op(h, dim, level, M.MHS_OP_EXACT, prec)   # tables built on first use
                M.mhs_level_write(h, dim, level, M.MHS_FIELD_U, prec, np.zeros(shape_l))
                n0 = M.mhs_kernel_launches()
                M.mhs_level_op(h, dim, level, M.MHS_OP_EXACT, prec)
                counts.append(M.mhs_kernel_launches() - n0)
                outs.append(_read(M, h, dim, level, M.MHS_FIELD_U, prec))
            assert counts == [1 if dim == 2 else 3, 5], (dim, level, counts)
            assert np.abs(outs[0]).max() > 0
            assert np.array_equal(outs[0], outs[1]), (dim, level, (lx, ly, lz), np.abs(outs[0] - outs[1]).max())
            checked += 1
    assert checked >= 2
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("exact_level", [1, 2])
def test_vcycle_exact_coarse_parity(M, exact_level, dim, prec):
    """One V(2,2)-cycle whose coarse-grid system on level 1 or 2 is solved
    exactly by the separable solver, against the oracle's V-cycle stopping at
    the same level with that system solved to rounding."""
    nx, ny, nz = 65, 33, 17
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=0.5, Lz=0.25)
    lx, ly, lz = M.mhs_level_shape(h, dim, exact_level)
    interior = (lx - 2) * (ly - 2) * ((lz - 2) if dim == 3 else 1)
    # sub-cycle only on the coarsest level, so that the cycle reaches exact_level
    M.mhs_set_options(h, flags=M.MHS_FLAG_POINT, sep_coarse=interior, cut64=1, cut32=1)
    rng = np.random.default_rng(13 + exact_level)
    shape = (nz, ny, nx) if dim == 3 else (ny, nx)
    u = rng.standard_normal(shape)
    f = rng.standard_normal(shape) * 100
    if dim == 2:
        u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = 0.0
    M.mhs_level_write(h, dim, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, dim, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    M.mhs_level_op(h, dim, 0, M.MHS_OP_VCYCLE, prec)
    got = _read(M, h, dim, 0, M.MHS_FIELD_U, prec)
    want = oracle.vcycle(pr, u, f, exact_level=exact_level)
    assert _rel(got, want) < (1e-11 if prec == 0 else 1e-5)
    # and not the cycle that descends to the coarsest level
    assert _rel(oracle.vcycle(pr, u, f), want) > 1e-7
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_vcycle_parity_3d(M, prec):
    nx, ny, nz = 33, 33, 17
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=1.0, Lz=0.5)
    rng = np.random.default_rng(11)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 100
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    M.mhs_level_op(h, 3, 0, M.MHS_OP_VCYCLE, prec)
    got = _read(M, h, 3, 0, M.MHS_FIELD_U, prec)
    want = oracle.vcycle(pr, u, f)
    assert _rel(got, want) < (1e-11 if prec == 0 else 1e-5)
    M.mhs_destroy(h)


@pytest.mark.parametrize("shape", [(17, 9, 13), (33, 17, 9), (65, 33, 33), (5, 5, 5), (129, 9, 65)])
def test_fused_sweep_equals_colour_passes_bitwise(M, shape):
    """The fused out-of-place red-black sweep (z-marching, shared-memory
    planes) computes every update from the same operands in the same order as
    the two in-place colour passes: the results are bitwise equal, over
    several sweeps, with non-zero Dirichlet data on every face."""
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + 3 * ny + 7 * nz)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 30
    out = []
    for flags in (0, M.MHS_FLAG_FUSED_SWEEP64):
        pr, h = _make(M, nx, ny, nz)
        M.mhs_set_options(h, flags=flags | M.MHS_FLAG_POINT)
        M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, 0, u)
        M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, 0, f)
        for _ in range(3):
            M.mhs_level_op(h, 3, 0, M.MHS_OP_SMOOTH, 0)
        out.append(_read(M, h, 3, 0, M.MHS_FIELD_U, 0))
        M.mhs_destroy(h)
    assert np.array_equal(out[0], out[1])
    assert _rel(out[1], oracle.rbgs3d(pr, u, f, 3)) < 1e-12


def test_fused_sweep_fp64_solve_matches_default(M):
    import torch
    pr, bz = S.linear_mhs(65, seed=17)
    res = []
    for flags in (0, M.MHS_FLAG_FUSED_SWEEP64):
        h = M.mhs_create(65, 65, 65, 1.0, 1.0, 1.0, pr["alpha"],
                         M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"]))
        M.mhs_set_options(h, flags=flags | M.MHS_FLAG_POINT)
        M.mhs_set_lower_bz(h, bz)
        info = M.mhs_solve(h, 1e-11, M.MHS_FP64)
        phi = np.zeros((65, 65, 65)); M.mhs_get_phi(h, phi)
        M.mhs_destroy(h)
        res.append((info, phi))
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("rows", [8, 16])
@pytest.mark.parametrize("shape", [(17, 9, 13), (33, 17, 9), (65, 33, 33), (5, 5, 5), (129, 9, 65), (129, 129, 65),
                                   (67, 19, 21), (131, 35, 11)])
def test_tma_sweep_equals_plain_fused_sweep_fp32(M, shape, rows):
    """FP32 sweeps with TMA-staged planes (mbarrier pipeline) give bitwise the
    results of the same sweep with plain global loads, over several sweeps
    and z-chunks, with non-zero Dirichlet data on every face, for tiles of 8
    and of 16 rows (ragged last tiles in x and y: 65 and 129 interior columns,
    17 and 33 interior rows)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(2 * nx + ny + nz)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 20
    out = []
    for flags in (0, M.MHS_FLAG_NO_TMA):
        pr, h = _make(M, nx, ny, nz)
        M.mhs_set_options(h, flags=flags | M.MHS_FLAG_POINT, fused_min=1, tma_rows=rows)
        M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, 1, u)
        M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, 1, f)
        for _ in range(5):
            M.mhs_level_op(h, 3, 0, M.MHS_OP_SMOOTH, 1)
        out.append(_read(M, h, 3, 0, M.MHS_FIELD_U, 1))
        M.mhs_destroy(h)
    assert np.array_equal(out[0], out[1])
    u32, f32 = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    assert _rel(out[0], oracle.rbgs3d(pr, u32, f32, 5)) < 1e-4


def test_tma_rows_other_than_8_or_16_are_rejected(M):
    pr, h = _make(M, 17, 9, 13)
    try:
        for rows in (4, 12, 32):
            with pytest.raises(M.MhsError):
                M.mhs_set_options(h, flags=M.MHS_FLAG_POINT, tma_rows=rows)
    finally:
        M.mhs_destroy(h)


@pytest.mark.parametrize("mode", [1, 0])
def test_out_of_place_sweeps_after_separable_solves(M, mode):
    """The twin array of the out-of-place sweeps is also scratch of the
    separable solver (exact coarse-grid solves, MHS_FLAG_SEPARABLE).  A solve
    that sweeps out of place on a handle that ran separable solves on the
    same levels before must equal that solve on a fresh handle bit for bit."""
    pr, bz = S.linear_mhs(65, seed=77)
    tol = 1e-10
    fused = dict(fused_min=1, flags=M.MHS_FLAG_POINT) if mode == 1 else \
        dict(flags=M.MHS_FLAG_POINT | M.MHS_FLAG_FUSED_SWEEP64)

    def phi_of(h):
        out = np.zeros((65, 65, 65))
        M.mhs_get_phi(h, out)
        return out

    def make():
        h = M.mhs_create(65, 65, 65, 1.0, 1.0, 1.0, pr["alpha"], M.xi_params(pr["xi_kind"], pr["xi_a"], pr["xi_kappa"]))
        M.mhs_set_lower_bz(h, bz)
        return h

    fresh = make()
    M.mhs_set_options(fresh, **fused)
    info_f = M.mhs_solve(fresh, tol, mode)
    want = phi_of(fresh)
    M.mhs_destroy(fresh)
    h = make()
    M.mhs_set_options(h, flags=M.MHS_FLAG_SEPARABLE)        # level 0's twin as scratch
    M.mhs_solve(h, tol, mode)
    M.mhs_set_options(h, sep_coarse=31 ** 3)                 # exact coarse-grid solve on 33^3: level 1's twin
    M.mhs_solve(h, tol, mode)
    M.mhs_set_options(h, **fused)
    info = M.mhs_solve(h, tol, mode)
    assert info["cycles_3d"] == info_f["cycles_3d"]
    assert np.array_equal(phi_of(h), want)
    M.mhs_destroy(h)


XI_STRONG = dict(xi_kind=1, xi_a=0.99, xi_kappa=0.5)   # 1 - xi(0) = 0.01: strong vertical coupling


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(17, 9, 13), (33, 17, 9), (65, 33, 33), (5, 5, 5), (129, 9, 65), (7, 67, 21),
                                   (9, 7, 53), (5, 9, 129), (7, 5, 201)])
def test_zline_sweep_parity(M, shape, prec):
    """Zebra z-line sweeps against the oracle's line sweeps, three sweeps with
    non-zero Dirichlet data on every face.  FP64 levels solve each column by
    one thread (Thomas elimination with precomputed pivots); FP32 levels by
    the partitioned solve, whose segment count follows nz: 1 (nz <= 25), 2, 4
    (nz 53: a ragged last segment of 9 planes), 8 (nz 129) and 16 (nz 201:
    segments of 12 planes, the last of 4)."""
    nx, ny, nz = shape
    pr, h = _make(M, nx, ny, nz, xi=XI_STRONG)
    M.mhs_set_options(h, flags=M.MHS_FLAG_ZLINE)
    rng = np.random.default_rng(5 * nx + ny + 3 * nz)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 30
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    for _ in range(3):
        M.mhs_level_op(h, 3, 0, M.MHS_OP_SMOOTH, prec)
    got = _read(M, h, 3, 0, M.MHS_FIELD_U, prec)
    want = oracle.zline3d(pr, u, f, 3)
    assert _rel(got, want) < (1e-12 if prec == 0 else 2e-5)
    M.mhs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("cut", [0, 40])
def test_zline_vcycle_parity(M, prec, cut):
    """One V(2,2)-cycle with z-line smoothing on every 3D level against the
    oracle's: with the default sub-cycle cut-off, and with a cut-off of 40
    nodes so that the global-memory line kernel runs on four levels."""
    nx, ny, nz = 65, 33, 33
    pr, h = _make(M, nx, ny, nz, Lx=1.0, Ly=0.5, Lz=0.5, xi=XI_STRONG)
    M.mhs_set_options(h, flags=M.MHS_FLAG_ZLINE, cut64=cut, cut32=cut, sep_coarse=-1)
    rng = np.random.default_rng(12)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx)) * 100
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_U, prec, u)
    M.mhs_level_write(h, 3, 0, M.MHS_FIELD_F, prec, f)
    if prec == 1:
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    M.mhs_level_op(h, 3, 0, M.MHS_OP_VCYCLE, prec)
    got = _read(M, h, 3, 0, M.MHS_FIELD_U, prec)
    want = oracle.vcycle(pr, u, f, smoother="zline")
    assert _rel(got, want) < (1e-11 if prec == 0 else 1e-5)
    M.mhs_destroy(h)
