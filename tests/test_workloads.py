"""The seeded input generators follow their stated recipe.

`workloads` is the one module the oracle, the tests and the benchmark share.
These checks hold it to the recipe its docstrings state: the counter-based
stream slices, which stream outputs each field takes, and the distributions
of the batched and served workloads (sizes, coefficient ranges, horizons,
arrival rate, the cell Peclet bound).
"""
import math

import numpy as np

import workloads as wl


def test_stream_slices_are_counter_based():
    """Any slice of a SplitMix64 stream equals the same slice of the full
    stream, so the v field's outputs [N, 2N) need no prefix."""
    full = wl.uniform01(17, 40)
    for off, cnt in ((0, 40), (7, 5), (39, 1), (20, 20)):
        assert np.array_equal(wl.uniform01(17, cnt, off), full[off:off + cnt])
    assert np.all((full >= 0.0) & (full < 1.0))
    # Box-Muller pairs: normal(seed, count, offset) takes uniform pairs from 2 * offset
    z = wl.normal(9, 10)
    assert np.array_equal(wl.normal(9, 4, 3), z[6:10])


def test_initial_data_takes_the_stated_outputs():
    """uniform data: equilibrium + amp (2 r - 1), u from outputs [0, N), v from
    [N, 2N), reshaped with x_1 fastest; normal data: amp * z likewise."""
    p = wl.schnakenberg_64().replace(n=(5, 3))
    u, v = wl.initial_data(p)
    N = 15
    ue, ve = wl.equilibrium(p.model, p.params)
    assert u.shape == (3, 5) and v.shape == (3, 5)
    ru = wl.uniform01(p.seed, N)
    rv = wl.uniform01(p.seed, N, N)
    assert np.array_equal(u.ravel(), ue + 0.01 * (2.0 * ru - 1.0))
    assert np.array_equal(v.ravel(), ve + 0.01 * (2.0 * rv - 1.0))
    assert u[1, 0] == u.ravel()[5]  # row-major (x_2, x_1): x_1 fastest
    q = wl.fhn_1024(n=4, nsteps=1)
    uq, vq = wl.initial_data(q)
    z = wl.normal(q.seed, 32)
    assert np.array_equal(uq.ravel(), 0.05 * z[:16])
    assert np.array_equal(vq.ravel(), 0.05 * z[16:])


def test_round_to_is_idempotent_and_exact_for_fp64():
    x = wl.initial_data(wl.fhn_1024(n=8, nsteps=1))[0]
    assert np.array_equal(wl.round_to(x, wl.FP64), x)
    r = wl.round_to(x, wl.FP32)
    assert np.array_equal(wl.round_to(r, wl.FP32), r)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -24


def _peclet(p):
    h = [(p.hi[m] - p.lo[m]) / (p.n[m] - 1) for m in range(p.d)]
    return max(abs(p.adv[c][m]) * h[m] / (2.0 * p.diff[c]) for c in range(2) for m in range(p.d))


def test_serving_stream_follows_recipe():
    reqs = wl.serving_stream(count=2000)
    t = np.array([a for a, _ in reqs])
    assert np.all(np.diff(t) > 0.0)
    # Poisson at 200/s: 2000 exponential gaps, mean within 5 standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 200.0 - 1.0) < 5.0 / math.sqrt(2000)
    d3 = sum(p.d == 3 for _, p in reqs)
    assert abs(d3 - 1000) < 5.0 * math.sqrt(2000 * 0.25)
    models = [p.model for _, p in reqs]
    for m in (wl.SCHNAKENBERG, wl.FHN, wl.BRUSSELATOR):
        assert abs(models.count(m) - 2000 / 3) < 5.0 * math.sqrt(2000 * 2 / 9)
    for i, (_, p) in enumerate(reqs):
        sides = wl.SERVE_SIDES_3D if p.d == 3 else wl.SERVE_SIDES_2D
        assert len(set(p.n)) == 1 and p.n[0] in sides
        assert 50 <= p.nsteps <= 1000
        assert p.seed == 100000 + i
        assert _peclet(p) < 1.0
        if p.model == wl.SCHNAKENBERG:
            assert 500.0 <= p.params[0] < 1500.0 and p.tau == wl.schnakenberg_tau(p.params[0])
            assert 0.5 <= p.diff[0] < 1.5 and 5.0 <= p.diff[1] < 15.0
        elif p.model == wl.FHN:
            assert 0.025 <= p.params[0] < 0.075 and p.tau == 1e-2 and p.hi[0] == 100.0
        else:
            assert 1.5 <= p.params[1] < 4.5 and p.tau == 1e-2
            assert 0.01 <= p.diff[0] < 0.03 and 0.05 <= p.diff[1] < 0.15
    # horizons cover the stated range
    steps = [p.nsteps for _, p in reqs]
    assert min(steps) < 70 and max(steps) > 980
    # the stream is a pure function of its seed; the rate only rescales time
    again = wl.serving_stream(count=50, rate=10.0)
    assert [p.n for _, p in again] == [p.n for _, p in reqs[:50]]
    assert np.allclose([a for a, _ in again], t[:50] * 20.0)


def test_batched_512_follows_recipe():
    probs = wl.batched_512()
    assert len(probs) == 512
    nf = 0
    for i, p in enumerate(probs):
        assert p.d == 2 and all(s in wl.BATCH_SIDES for s in p.n)
        assert p.seed == 1000 + i and p.nsteps == 100
        assert p.diff[0] == 1.0 and 5.0 <= p.diff[1] < 40.0
        if p.model == wl.SCHNAKENBERG:
            g = p.params[0]
            assert 100.0 <= g < 2000.0
            assert math.isclose(p.tau, min(max(0.125 / g, 6.25e-5), 1.25e-3), rel_tol=1e-14)
            assert p.hi == (1.0, 1.0)
        else:
            assert p.model == wl.FHN and p.tau == 1e-2 and p.hi == (100.0, 100.0)
            nf += 1
    assert abs(nf - 256) < 5.0 * math.sqrt(512 * 0.25)
    # non-square grids occur
    assert any(p.n[0] != p.n[1] for p in probs)
