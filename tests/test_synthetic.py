"""The seeded synthetic inputs that the oracle tests, the GPU parity tests and
the benchmark share: the splitmix64 stream, the Gaussian-source magnetograms
(B_z = B_0 exp(-r^2 / l^2), Sect. 3.1) and the workload recipes."""
import numpy as np

import synthetic as S


def test_splitmix64_reference_outputs():
    """The first outputs of splitmix64 from state 0, as published with the
    generator's reference implementation."""
    r = S.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_draws():
    a, b = S.SplitMix64(1307), S.SplitMix64(1307)
    xs = [a.uniform() for _ in range(100_000)]
    assert xs[:100] == [b.uniform() for _ in range(100)]
    assert min(xs) >= 0.0 and max(xs) < 1.0
    assert abs(np.mean(xs) - 0.5) < 0.005
    assert abs(np.var(xs) - 1.0 / 12.0) < 0.002
    r = S.SplitMix64(7)
    assert all(-2.0 <= r.uniform(-2.0, 3.0) < 3.0 for _ in range(1000))


def test_random_magnetogram_is_flux_balanced_and_reproducible():
    for n, seed in ((33, 3), (129, 1307), (65, 9000)):
        bz = S.magnetogram_random(n, n, 1.0, 1.0, seed=seed)
        assert bz.shape == (n, n)
        assert abs(bz.sum()) <= 1e-12 * np.abs(bz).sum()
        assert np.array_equal(bz, S.magnetogram_random(n, n, 1.0, 1.0, seed=seed))
        assert bz.max() > 0 > bz.min()
    assert not np.array_equal(S.magnetogram_random(33, 33, seed=1), S.magnetogram_random(33, 33, seed=2))


def test_random_spot_parameters():
    for seed in range(50):
        for s in S.random_spots(seed):
            assert -1.0 <= s.amp < 1.0
            assert 0.03 <= s.sigma < 0.1
            assert 0.15 <= s.x0 < 0.85 and 0.15 <= s.y0 < 0.85


def test_potential_field_pair_is_antisymmetric():
    pr, bz = S.potential_field_33()
    assert pr["alpha"] == 0.0 and pr["xi_kind"] == 0 and (pr["nx"], pr["ny"], pr["nz"]) == (33, 33, 33)
    assert np.abs(bz + bz[:, ::-1]).max() <= 1e-15
    assert abs(bz.sum()) <= 1e-12
    j = 16   # the row through both centres: the +1 source peaks at x = 0.35 (node 11.2)
    assert np.argmax(bz[j]) == 11 and np.argmin(bz[j]) == 21


def test_batched_instances_recipe():
    inst = S.batched_instances(256)
    assert len(inst) == 256
    shapes = [(33, 33, 1.0), (65, 65, 1.0), (129, 129, 1.0), (129, 65, 0.5)]
    for i, d in enumerate(inst):
        assert (d["n"], d["nz"], d["Lz"]) == shapes[i % 4]
        assert 0.0 <= d["alpha"] < 0.8 and 0.0 <= d["a"] < 1.0 and 0.5 <= d["kappa"] < 2.0
        assert d["bz"].shape == (d["n"], d["n"])
        pr = S.batched_problem(d)
        assert (pr["nx"], pr["ny"], pr["nz"], pr["Lz"]) == (d["n"], d["n"], d["nz"], d["Lz"])
        assert pr["xi_kind"] == 1 and pr["xi_a"] == d["a"] and pr["xi_kappa"] == d["kappa"]
    again = S.batched_instances(8)
    assert all(np.array_equal(a["bz"], b["bz"]) and a["alpha"] == b["alpha"] for a, b in zip(inst[:8], again))


def test_linear_mhs_workload_and_unknowns():
    pr, bz = S.linear_mhs(129)
    assert (pr["alpha"], pr["xi_a"], pr["xi_kappa"], pr["xi_kind"]) == (0.5, 0.5, 1.0, 1)
    assert bz.shape == (129, 129)
    assert S.unknowns(pr) == 127 ** 3 + 127 ** 2
    pr2, _ = S.linear_mhs(513, nz=257, Lz=0.5)
    assert (pr2["nz"], pr2["Lz"]) == (257, 0.5)
    assert S.unknowns(pr2) == 511 * 511 * 255 + 511 * 511
