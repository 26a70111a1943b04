"""The seeded synthetic inputs (workloads.py) follow their stated recipes:
sizes, cross sections, moment shapes, sources, boundaries and multigrid
set-up of each workload, and the same seed gives the same problem (CPU)."""
import numpy as np
import pytest

import workloads as W


def _unknowns(p):
    s = 2 ** p["dim"]
    a = 3 if p["basis"] == "lin" else 1
    return int(np.prod(p["ncell"])) * s * 8 * 4 ** p["level"] * a


def _same(p, q):
    assert p.keys() == q.keys()
    for k in p:
        if isinstance(p[k], np.ndarray):
            assert np.array_equal(p[k], q[k]), k
        else:
            assert p[k] == q[k], k


def _source_volume(p):
    h = [(p["hi"][e] - p["lo"][e]) / p["ncell"][e] for e in range(p["dim"])]
    return float(p["q"].sum() * np.prod(h))


@pytest.mark.parametrize("make", [W.config1_square16, W.config2_checkerboard,
                                  lambda: W.config4_batch(nprob=8),
                                  lambda: W.random_problem(3, (3, 2, 4), 1, 5, 7)],
                         ids=["config1", "config2", "config4", "random"])
def test_the_same_seed_gives_the_same_problem(make):
    a, b = make(), make()
    if isinstance(a, list):
        for p, q in zip(a, b):
            _same(p, q)
    else:
        _same(a, b)


def test_config1_square16():
    p = W.config1_square16()
    assert p["ncell"] == (16, 16) and p["level"] == 1 and p["N"] == 8
    assert np.all(p["sigma_t"] == 1.0) and np.all(p["sigma_s"] == 0.9)
    assert np.allclose(p["fmom"], 0.8 ** np.arange(9))
    assert abs(_source_volume(p) - 0.25 ** 2) < 1e-15        # centred 0.25 x 0.25 square
    assert p["mg"]["nlevels"] == 2 and p["mg"]["Nr"] == [8, 4]


def test_config2_checkerboard():
    p = W.config2_checkerboard()
    n = 128
    assert p["ncell"] == (n, n) and p["level"] == 3 and p["N"] == 16
    st = p["sigma_t"].reshape(n, n)
    # constant on every 16 x 16 tile, both materials present
    tiles = st.reshape(8, 16, 8, 16)
    assert np.all(tiles == tiles[:, :1, :, :1])
    assert set(np.unique(st)) == {1.0, 10.0}
    ratio = p["sigma_s"] / p["sigma_t"]
    assert np.allclose(ratio[p["sigma_t"] == 1.0], 0.5)
    assert np.allclose(ratio[p["sigma_t"] == 10.0], 0.99)
    assert np.allclose(p["fmom"], 0.9 ** np.arange(17))
    assert abs(_source_volume(p) - 0.25 ** 2) < 1e-15
    assert p["mg"]["Nr"] == [16, 4, 4]
    assert _unknowns(p) == 128 * 128 * 4 * 512 * 3         # 1.01e8


def test_config3_cube():
    p = W.config3_cube(n=16)                               # same recipe, fewer cells
    st = p["sigma_t"]
    assert p["ncell"] == (16, 16, 16) and p["level"] == 2 and p["N"] == 32
    assert np.allclose(p["sigma_s"], 0.9 * st)
    assert len(np.unique(st)) == st.size                   # a material per cell
    assert abs(np.log(st).mean()) < 0.05 and abs(np.log(st).std() - 0.5) < 0.05
    assert np.allclose(p["fmom"], 0.95 ** np.arange(33))
    assert abs(_source_volume(p) - 0.25 ** 3) < 1e-15


def test_config4_batch():
    ps = W.config4_batch()
    assert len(ps) == 256
    ns = np.array([p["ncell"][0] for p in ps])
    lv = np.array([p["level"] for p in ps])
    assert ns.min() >= 16 and ns.max() <= 96 and len(np.unique(ns)) > 40
    assert set(lv) == {1, 2, 3}
    for p in ps:
        n, L = p["ncell"][0], p["level"]
        assert p["ncell"] == (n, n) and p["N"] == 2 * L + 4
        ratio = p["sigma_s"] / p["sigma_t"]
        assert np.ptp(ratio) < 1e-12 and 0.5 <= ratio[0] <= 0.95
        g = p["fmom"][1]
        assert 0.7 <= g <= 0.95 and np.allclose(p["fmom"], g ** np.arange(p["N"] + 1))
        assert p["mg"]["nlevels"] == L and p["mg"]["Nr"][1:] == [min(p["N"], 4)] * (L - 1)
    total = sum(_unknowns(p) for p in ps)
    assert 2.0e9 < total < 3.2e9                           # "about 2.5e9 DOF in total"


def test_config5_beam():
    p = W.config5_beam()
    assert p["ncell"] == (256, 256) and p["level"] == 4 and p["N"] == 64
    assert np.all(p["sigma_t"] == 5.0) and np.all(p["sigma_s"] == 4.95)
    assert np.allclose(p["fmom"], 0.98 ** np.arange(65))
    assert not p["q"].any()
    assert p["boundary"] == [(2, 1.0), (0, 0.0), (0, 0.0), (0, 0.0)]   # unit beam, low-x edge
    assert p["mg"]["nlevels"] == 4 and p["mg"]["Nr"] == [64, 12, 12, 12]
    assert _unknowns(p) == 256 * 256 * 4 * 2048 * 3        # 1.61e9


@pytest.mark.parametrize("N", [4, 8, 16])
def test_table1_cube(N):
    p = W.table1_cube(N, n=6)                              # same recipe, fewer cells
    assert p["hi"] == (5.0, 5.0, 5.0) and p["level"] == 3
    s0 = N * (N + 1) / 2
    assert np.all(p["sigma_t"] == s0) and np.all(p["sigma_s"] == s0)
    sn = s0 * p["fmom"]
    assert abs((p["sigma_t"][0] - sn[1]) - 1.0) < 1e-12    # transport cross section 1
    assert np.all(p["q"] == 1.0)
    assert p["mg"]["nlevels"] == 4
