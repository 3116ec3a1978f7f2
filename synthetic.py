"""Seeded synthetic inputs for the linear MHS solver.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It holds no arithmetic of the solution method itself: it only
draws random numbers and evaluates the Gaussian source model that the paper
uses to prescribe the normal field on the photosphere (Sect. 3.1,
B_z(r) = B_0 exp(-r^2 / l^2)).

Random numbers come from splitmix64 (G. Steele, D. Lea, C. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser
constants are the published ones), converted to doubles in [0, 1) from the top
53 bits.  Everything is plain Python / numpy so both sides of a comparison can
call it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream: state += golden gamma; output = mix(state)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u


@dataclasses.dataclass(frozen=True)
class Spot:
    amp: float      # B_0 of the source (signed)
    x0: float
    y0: float
    sigma: float    # the paper's source width l


def node_coords(n: int, length: float, origin: float = 0.0) -> np.ndarray:
    """Vertex-centred node coordinates origin + i * length / (n - 1)."""
    return origin + np.arange(n, dtype=np.float64) * (length / (n - 1))


def spots_field(nx: int, ny: int, Lx: float, Ly: float, spots, x_origin: float = 0.0,
                y_origin: float = 0.0) -> np.ndarray:
    """Sum of Gaussian sources on the node grid, shape [ny][nx] (x fastest)."""
    x = node_coords(nx, Lx, x_origin)[None, :]
    y = node_coords(ny, Ly, y_origin)[:, None]
    bz = np.zeros((ny, nx), dtype=np.float64)
    for s in spots:
        bz += s.amp * np.exp(-((x - s.x0) ** 2 + (y - s.y0) ** 2) / (s.sigma ** 2))
    return bz


def random_spots(seed: int, n_spots: int = 8, amp=(-1.0, 1.0), sigma=(0.03, 0.1),
                 centre=(0.15, 0.85)):
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_spots):
        a = rng.uniform(*amp)
        s = rng.uniform(*sigma)
        cx = rng.uniform(*centre)
        cy = rng.uniform(*centre)
        out.append(Spot(a, cx, cy, s))
    return out


def flux_balanced_spots(nx: int, ny: int, Lx: float, Ly: float, spots):
    """Scale the negative sources so that the node sum of B_z vanishes.

    Positive and negative node fluxes are summed per source sign; every
    negative amplitude is multiplied by Phi_plus / |Phi_minus|.  Without a
    source of either sign the list is returned unchanged.
    """
    pos = [s for s in spots if s.amp > 0]
    neg = [s for s in spots if s.amp < 0]
    if not pos or not neg:
        return list(spots)
    phi_p = spots_field(nx, ny, Lx, Ly, pos).sum()
    phi_m = spots_field(nx, ny, Lx, Ly, neg).sum()
    k = phi_p / abs(phi_m)
    return pos + [Spot(s.amp * k, s.x0, s.y0, s.sigma) for s in neg]


def magnetogram_random(nx: int, ny: int, Lx: float = 1.0, Ly: float = 1.0, seed: int = 1307,
                       n_spots: int = 8) -> np.ndarray:
    """Flux-balanced random multi-spot magnetogram on [0,Lx]x[0,Ly].

    Spot amplitudes ~ U[-1,1], widths ~ U[0.03,0.1], centres ~ U[0.15,0.85]^2
    (scaled by the domain size), drawn from splitmix64(seed).
    """
    sp = random_spots(seed, n_spots)
    sp = [Spot(s.amp, s.x0 * Lx, s.y0 * Ly, s.sigma * min(Lx, Ly)) for s in sp]
    sp = flux_balanced_spots(nx, ny, Lx, Ly, sp)
    return spots_field(nx, ny, Lx, Ly, sp)


def magnetogram_pair(nx: int, ny: int, sigma: float = 0.08) -> np.ndarray:
    """+1 spot at (0.35,0.5) and -1 spot at (0.65,0.5) on [0,1]^2.

    The pair is antisymmetric under x -> 1 - x, which on an odd node count maps
    node i to node nx-1-i, so its node sum vanishes up to rounding.
    """
    return spots_field(nx, ny, 1.0, 1.0, [Spot(1.0, 0.35, 0.5, sigma), Spot(-1.0, 0.65, 0.5, sigma)])


def magnetogram_three_sources(nx: int, ny: int) -> np.ndarray:
    """Force-free example of Sect. 3.1: domain [-5.5,5.5]^2, l = 0.3, one +1 source
    at (1.5,1.5) and two -0.5 sources at (-1.5,-1.5), (1.5,-1.5)."""
    sp = [Spot(1.0, 1.5, 1.5, 0.3), Spot(-0.5, -1.5, -1.5, 0.3), Spot(-0.5, 1.5, -1.5, 0.3)]
    return spots_field(nx, ny, 11.0, 11.0, sp, -5.5, -5.5)


def magnetogram_mode(nx: int, ny: int, Lx: float, Ly: float, m: int = 1, n: int = 1) -> np.ndarray:
    """sin(m pi x / Lx) sin(n pi y / Ly) sampled on the nodes."""
    x = node_coords(nx, Lx)[None, :]
    y = node_coords(ny, Ly)[:, None]
    return np.sin(m * math.pi * x / Lx) * np.sin(n * math.pi * y / Ly)


# ----------------------------------------------------------------------------
# Workload descriptions (sizes, physics parameters, seeds).  A "problem" is a
# plain dict so that both the oracle and the GPU binding can read it.
# ----------------------------------------------------------------------------

def problem(nx, ny, nz, Lx=1.0, Ly=1.0, Lz=1.0, alpha=0.0, xi_kind=0, xi_a=0.0, xi_kappa=0.0,
            xi_b=0.0, xi_omega=0.0, g=1.0, mu0=0.5, T_cor=150.0, z1=5.0, z2=10.0):
    return dict(nx=nx, ny=ny, nz=nz, Lx=Lx, Ly=Ly, Lz=Lz, alpha=alpha, xi_kind=xi_kind,
                xi_a=xi_a, xi_kappa=xi_kappa, xi_b=xi_b, xi_omega=xi_omega, g=g, mu0=mu0,
                T_cor=T_cor, z1=z1, z2=z2)


def potential_field_33():
    """Potential-field limit (xi = 0, alpha = 0) on 33^3 nodes of [0,1]^3 with the
    antisymmetric +/-1 spot pair (sigma = 0.08)."""
    pr = problem(33, 33, 33)
    return pr, magnetogram_pair(33, 33, 0.08)


def linear_mhs(n=129, seed=1307, alpha=0.5, a=0.5, kappa=1.0, nz=None, Lz=None):
    """Linear MHS workload: alpha = 0.5, xi(z) = a exp(-kappa z), 8 flux-balanced
    random spots; n^3 nodes on [0,1]^3 unless nz / Lz are given."""
    nz = n if nz is None else nz
    Lz = 1.0 if Lz is None else Lz
    pr = problem(n, n, nz, 1.0, 1.0, Lz, alpha=alpha, xi_kind=1, xi_a=a, xi_kappa=kappa)
    return pr, magnetogram_random(n, n, 1.0, 1.0, seed)


def unknowns(pr) -> int:
    """3D interior unknowns plus the 2D lower-boundary interior unknowns."""
    nx, ny, nz = pr["nx"], pr["ny"], pr["nz"]
    return (nx - 2) * (ny - 2) * (nz - 2) + (nx - 2) * (ny - 2)


def batched_instances(count=256):
    """The uneven batch: grids 33^3, 65^3, 129^3 on [0,1]^3 and 129 x 129 x 65 on
    [0,1]^2 x [0,0.5] in turn; alpha ~ U[0,0.8], xi = a exp(-kappa z) with
    a ~ U[0,1), kappa ~ U[0.5,2], 8-spot magnetogram; instance i draws from
    splitmix64(1000 + i)."""
    shapes = [(33, 33, 1.0), (65, 65, 1.0), (129, 129, 1.0), (129, 65, 0.5)]
    inst = []
    for i in range(count):
        n, nz, Lz = shapes[i % 4]
        rng = SplitMix64(1000 + i)
        alpha, a, kappa = rng.uniform(0.0, 0.8), rng.uniform(0.0, 1.0), rng.uniform(0.5, 2.0)
        inst.append(dict(n=n, nz=nz, Lz=Lz, alpha=alpha, a=a, kappa=kappa,
                         bz=magnetogram_random(n, n, seed=1000 + i)))
    return inst


def batched_problem(d):
    """The problem dict of one batched instance."""
    return problem(d["n"], d["n"], d["nz"], 1.0, 1.0, d["Lz"], alpha=d["alpha"], xi_kind=1,
                   xi_a=d["a"], xi_kappa=d["kappa"])
