"""The seeded input generators (CPU only): the counter-based SplitMix64 stream
against its published outputs, determinism and independence of streams, and
the structure every workload recipe promises (dominance, symmetry, band
widths, value ranges)."""
import numpy as np

import synthetic


def test_splitmix64_published_outputs():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 1234567: the first five
    # outputs of the reference implementation.
    with np.errstate(over="ignore"):
        z = np.uint64(1234567) + np.arange(1, 6, dtype=np.uint64) * synthetic.GAMMA
    assert [int(v) for v in synthetic._mix64(z)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]


def test_streams_are_counter_based_and_independent():
    a = synthetic.uniform01(5, 0, 0, 1000)
    assert np.array_equal(a[300:700], synthetic.uniform01(5, 0, 300, 400))  # any window, same values
    assert np.all((a >= 0.0) & (a < 1.0))
    assert not np.array_equal(a, synthetic.uniform01(5, 1, 0, 1000))
    assert not np.array_equal(a, synthetic.uniform01(6, 0, 0, 1000))
    assert abs(a.mean() - 0.5) < 0.05


def test_dense_dd_is_strictly_row_dominant():
    for n, w in ((1, 0.9), (7, 0.5), (300, 0.9)):
        a = synthetic.dense_dd(n, w, 11 + n)
        assert np.array_equal(np.diag(a), np.ones(n))
        off = np.abs(a).sum(axis=1) - 1.0
        assert np.all(off <= w)
        assert np.array_equal(a, synthetic.dense_dd(n, w, 11 + n))
    # chunked generation draws the same values as one pass
    a = synthetic.dense_dd(40, 0.9, 3)
    u = synthetic.uniform01(3, synthetic.STREAM_A, 0, 1600).reshape(40, 40)
    off = ~np.eye(40, dtype=bool)
    assert np.array_equal(a[off], ((2.0 * u - 1.0) * (0.9 / 39))[off])


def test_laplacian_bands():
    ab, kl, ku = synthetic.laplacian_band(9)
    a = synthetic.band_to_dense(ab, kl, ku)
    assert kl == ku == 9 and np.array_equal(a, a.T)
    assert np.all(np.diag(a) == 4.1) and np.all(np.abs(a).sum(axis=1) - 4.1 <= 4.0)
    assert a[8, 9] == 0.0 and a[9, 8] == 0.0  # no neighbour across the end of a grid row
    assert np.array_equal(synthetic.dense_to_band(a, kl, ku), ab)
    for r in (1, 5, 12):
        ab, kl, ku = synthetic.laplacian_disc_band(r)
        a = synthetic.band_to_dense(ab, kl, ku)
        ys, xs = np.mgrid[-r:r + 1, -r:r + 1]
        n = int((xs * xs + ys * ys <= r * r).sum())
        assert a.shape == (n, n) and np.array_equal(a, a.T)
        deg = (a != 0).sum(axis=1) - 1
        assert deg.max() <= 4 and np.all(np.abs(a).sum(axis=1) - 4.1 < 4.1)
        i, j = np.nonzero(np.triu(a, 1))
        assert kl == ku == int((j - i).max())  # the widest band the numbering needs
        assert np.array_equal(synthetic.dense_to_band(a, kl, ku), ab)


def test_band_rhs_is_the_product():
    ab, kl, ku = synthetic.laplacian_disc_band(6)
    x = synthetic.planted_x(ab.shape[0], 3, 4)
    np.testing.assert_allclose(synthetic.band_rhs(ab, kl, ku, x), synthetic.band_to_dense(ab, kl, ku) @ x,
                               rtol=0, atol=1e-14)


def test_workload_metadata():
    ns, rs = synthetic.config3_sizes()
    assert ns.min() >= 16 and ns.max() <= 512 and rs.min() >= 1 and rs.max() <= 4
    p = synthetic.pick_indices(3, 100, [7, 1000])
    assert p.shape == (100, 2) and p[:, 0].max() < 7 and p[:, 1].max() < 1000 and p.min() >= 0
    g = synthetic.gaussian(1, synthetic.STREAM_W, (4000,))
    assert abs(g.mean()) < 0.1 and abs(g.std() - 1.0) < 0.1
