"""The seeded synthetic inputs (no GPU): sizes, level counts, coefficient fields and right-hand sides
of the five benchmark configurations and the paper-shaped variant, as the configurations state them."""
import numpy as np

from paper_1402_3545_gb300 import workloads


def test_configuration_sizes_and_levels():
    s, m, x, t = workloads.small(), workloads.mid(), workloads.mixed(), workloads.learned_target()
    assert (s.nx, s.ny, s.nz, s.nlevels) == (64, 64, 64, 4)          # 64 -> 8
    assert (m.nx, m.ny, m.nz, m.nlevels) == (512, 512, 128, 7)       # 512 -> 8
    assert (x.nx, x.ny, x.nz, x.nlevels) == (1024, 1024, 128, 8)
    assert (t.nx, t.ny, t.nz, t.nlevels) == (2048, 2048, 64, 9)
    for p in (s, m, x, t):
        assert p.omega2 == 1e-2 and p.hx == 1.0 / p.nx and p.hy == 1.0 / p.ny and p.hz == 1.0 / p.nz
    assert s.lambda2 == 1e3 and x.lambda2 == 1e4 and t.lambda2 == 1e3
    assert m.n == 512 * 512 * 128 and x.n == 134217728 and t.n == 268435456


def test_varying_lambda_field():
    """lambda^2(x, y) = 1e3 (1 + 0.5 sin 2 pi x cos 2 pi y) at cell centres: check points where the
    sine and cosine take simple values, the extremes 500 and 1500, and the mean 1e3."""
    nx = ny = 8
    lam = workloads.lambda2_varying(nx, ny)  # (ny, nx)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    for j in range(ny):
        for i in range(nx):
            ref = 1e3 * (1.0 + 0.5 * np.sin(2 * np.pi * x[i]) * np.cos(2 * np.pi * y[j]))
            assert abs(lam[j, i] - ref) < 1e-9
    big = workloads.lambda2_varying(512, 512)
    assert 500.0 <= big.min() < 501.0 and 1499.0 < big.max() <= 1500.0
    assert abs(big.mean() - 1e3) < 1e-9
    # rows are y, columns x: on a 4 x 4 grid cell (j, i) = (1, 0) sits at x = 1/8, y = 3/8, where
    # sin 2 pi x = cos(pi / 4) and cos 2 pi y = -cos(pi / 4): 1e3 (1 - 0.5 / 2) = 750
    lam4 = workloads.lambda2_varying(4, 4)
    assert abs(lam4[1, 0] - 750.0) < 1e-9 and abs(lam4[0, 1] - 1250.0) < 1e-9


def test_right_hand_sides():
    s = workloads.small()
    f = s.rhs()
    assert f.shape == (64, 64, 64) and abs(f.mean()) < 1e-15 and np.abs(f).max() <= 2.0
    g = workloads.make_rhs(64, 64, 64, 0, "uniform")
    assert np.allclose(f, g - g.mean()) and g.min() >= -1.0 and g.max() <= 1.0
    m = workloads.make_rhs(32, 32, 16, 0, "normal")
    assert abs(m.mean()) < 0.05 and abs(m.std() - 1.0) < 0.05
    # seeded: the same draw twice, another seed another draw
    assert np.array_equal(m, workloads.make_rhs(32, 32, 16, 0, "normal"))
    assert not np.array_equal(m, workloads.make_rhs(32, 32, 16, 1, "normal"))


def test_batched_draw():
    probs = workloads.batched()
    assert len(probs) == 64
    cells = 0
    for b, p in enumerate(probs):
        assert p.nx in (64, 128, 256, 512) and p.ny in (64, 128, 256, 512) and p.nz in (32, 64, 128)
        assert 1e2 <= p.lambda2 <= 1e4 and p.seed == 1000 + b
        assert p.hx == p.hy == 1.0 / max(p.nx, p.ny)
        assert p.nlevels == workloads.levels_to_8(p.nx, p.ny)
        cells += p.n
    assert cells == 286654464  # the draw the batched benchmark runs
    # log-uniform lambda^2: about half below 1e3
    below = sum(p.lambda2 < 1e3 for p in probs)
    assert 20 <= below <= 44


def test_levels_to_8():
    assert workloads.levels_to_8(64, 64) == 4 and workloads.levels_to_8(512, 512) == 7
    assert workloads.levels_to_8(512, 64) == 7   # elongated: the long side keeps coarsening to 8
    # 96 x 8 -> 48 x 4 -> 24 x 2 -> 12 x 1: stops when a side turns odd
    assert workloads.levels_to_8(96, 8) == 4
    assert workloads.levels_to_8(192, 96) == 6   # -> 6 x 3
    assert workloads.levels_to_8(8, 8) == 1
