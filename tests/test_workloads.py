"""Seeded input generators (no method arithmetic): SplitMix64 against its
published outputs, and the shapes / ranges of the synthetic workloads."""
import os

import numpy as np

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_published_outputs():
    lines = [l.strip() for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt"))
             if l.strip() and not l.startswith("#")]
    want = [int(x, 16) for x in lines]
    got = [int(v) for v in workloads.splitmix64(0, 4)]
    assert got == want
    st = workloads.Stream(0)
    assert [int(v) for v in st.raw(2)] + [int(v) for v in st.raw(2)] == want


def test_uniform_and_normal_moments():
    u = workloads.Stream(11).uniform(200000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    z = workloads.Stream(12).normal(200001)
    assert z.shape == (200001,)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1) < 1e-2


def test_lattice32_case():
    c = workloads.lattice32()
    assert c["sigma"].shape == (32, 32)
    s = c["sigma"]
    assert 1.0 <= s.min() and s.max() <= 100.0
    # piecewise constant on 4x4 blocks
    assert np.all(s[::4, ::4].repeat(4, 0).repeat(4, 1) == s)
    assert (c["r"], c["n_polar"], c["n_azim"], c["steps"]) == (6, 8, 16, 10)


def test_checker256_case():
    c = workloads.checker256()
    vals = set(np.unique(c["sigma"]).tolist())
    assert vals <= {0.1, 100.0} and len(vals) == 2
    assert (c["r"], c["n_polar"] * c["n_azim"]) == (16, 512)


def test_lognormal_sigma_small():
    s = workloads.lognormal_sigma(64, 2)
    z = (np.log(s) - np.log(5.0)) / 1.5
    assert abs(z.mean()) < 1e-12 and abs(z.std() - 1.0) < 1e-12


def test_batch_and_served_streams():
    b = workloads.batch64(n=8, steps=2)
    assert len(b) == 8
    for c in b:
        assert c["nx"] in (64, 128, 256, 512) and c["r"] in (8, 16, 24, 32)
        assert c["n_polar"] * c["n_azim"] in (128, 256, 512, 1024)
    reqs = workloads.served_requests(n=100)
    t = [a for a, _ in reqs]
    assert all(t[i] < t[i + 1] for i in range(len(t) - 1))
    gaps = np.diff([0.0] + t)
    assert 0.02 < gaps.mean() < 0.09
    for _, r in reqs:
        assert 128 <= r["side"] <= 1024 and r["r"] in (8, 16, 32) and 50 <= r["steps"] <= 200
