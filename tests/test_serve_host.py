"""Host logic of the serving layer that needs no GPU: the choice of FC
continuation lengths (smooth_n_cont) and the device footprint estimate."""
import pytest

serve = pytest.importorskip("paper_2606_06247_gb300.serve")


def _factors(m, primes):
    for q in primes:
        while m % q == 0:
            m //= q
    return m == 1


def test_smooth_n_cont_keeps_25_where_the_engine_is_direct():
    for n in (40, 96, 128, 200, 600):  # 65 = 5 13, 121 = 11^2, 153 = 9 17, 225, 625
        assert serve.smooth_n_cont(n) == 25


def test_smooth_n_cont_picks_the_nearest_7_smooth_length():
    expect = {64: 26, 256: 24, 512: 28, 1024: 26, 161: 28, 16: 24, 48: 24}
    for n, c in expect.items():
        assert serve.smooth_n_cont(n) == c
    for n in range(8, 2049):
        c = serve.smooth_n_cont(n)
        assert 20 <= c <= 40
        if c != 25:
            assert _factors(n + c, (2, 3, 5, 7))
            # no length in range nearer to 25, nor as near and smaller, qualifies
            d = abs(c - 25)
            nearer = [cc for cc in range(20, 41) if abs(cc - 25) < d or (abs(cc - 25) == d and cc < c)]
            assert not any(_factors(n + cc, (2, 3, 5, 7)) for cc in nearer if cc != 25)
        else:
            assert _factors(n + 25, (2, 3, 5, 7, 11, 13, 17)) or all(
                not _factors(n + cc, (2, 3, 5, 7)) for cc in range(20, 41))


def test_footprint_counts_the_continuation():
    # 3D: the spectra hold (n + C) / 2 + 1 rows of n^2 columns
    a = serve.footprint_bytes(16, 2, "f32x2", True, 24)
    b = serve.footprint_bytes(16, 2, "f32x2", True, 40)
    assert b > a > 0
