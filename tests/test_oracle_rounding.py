"""Why the FP64 bar for B_z and rho on the 513 x 513 x 257 grid is 1e-9.

B_z and rho are second and third differences of P (Sect. 2.2, eqs. b_iden,
density), so the rounding of P reaches them amplified by up to h^-2 and h^-3.
Two FP64 solutions of the same discrete equations that differ only by
rounding - the oracle's multigrid and the separable direct solver - are
compared on the benchmark's non-cubic family (n x n x (n+1)/2 nodes on
[0,1]^2 x [0,0.5], alpha = 0.5, xi = 0.5 exp(-z)) at h = 1/64, 1/128, 1/256.
Stopping the multigrid at 1e-13 or 1e-14 gives the same rho difference, so
the difference is rounding, not iteration error; it grows by about h^-3 per
halving of h.  Extrapolated one halving further, to the 513 x 513 x 257 grid
(h = 1/512), rounding alone puts rho at least half of 1e-10 away from the
direct solution: a 1e-10 bar there leaves no room for the solve error, and
the tests hold B_z and rho on that grid to 1e-9."""
import numpy as np

import oracle
import synthetic as S
from oracle import exact


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_rho_rounding_floor_grows_like_h_cubed():
    d = {}
    for n in (65, 129, 257):
        pr, bz = S.linear_mhs(n, nz=(n - 1) // 2 + 1, Lz=0.5)
        Fe = oracle.fields(pr, exact.exact_solution(pr, bz))
        P14, i14 = oracle.solve(pr, bz, 1e-14, 1e-14)
        assert i14["rel_res_3d"] < 1e-13 and i14["rel_res_2d"] < 1e-12, i14   # 2D: its rounding floor
        d[n] = _rel(oracle.fields(pr, P14)["rho"], Fe["rho"])
        if n == 257:
            P13, i13 = oracle.solve(pr, bz, 1e-13, 1e-13)
            d13 = _rel(oracle.fields(pr, P13)["rho"], Fe["rho"])
            assert 1 / 1.5 < d13 / d[n] < 1.5, (d13, d[n])   # rounding, not iteration error
    r1, r2 = d[129] / d[65], d[257] / d[129]
    assert r1 > 6 and r2 > 6, d                            # about h^-3 per halving
    predicted_513 = d[257] * (d[257] / d[65]) ** 0.5        # one more halving at the measured mean rate
    assert predicted_513 > 0.5e-10, (d, predicted_513)
