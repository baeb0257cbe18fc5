"""The closed-form default tile size (the paper's idea of fitting tuned
parameters as quadratics in log10 n): the committed header holds the fit of
the committed tuned tables, the fit reproduces the GA's winners at the tuned
sizes, and the library's resolved default follows it (host only, no GPU)."""
import math

import pytest
import torch

from paper_2505_18681_gb300 import closed_form as cf


def test_header_is_the_fit_of_the_committed_tables():
    with open(cf.HEADER) as f:
        assert f.read() == cf.header_text(cf.fits_from_tables()), \
            "csrc/closed_form.h is stale: run python -m paper_2505_18681_gb300.closed_form --write"


@pytest.mark.parametrize("w", [4, 8])
def test_fit_reproduces_the_tuned_winners(w):
    pts = cf.table_points(cf.TABLES[w])
    assert len(pts) >= 2
    coefs, rng = cf.fits_from_tables()[w]
    for L, log2_tile in pts:
        n = int(round(10 ** L))
        got = cf.nearest_shape(w, cf.evaluate(coefs, rng, n))
        assert math.log2(got[0] * got[1]) == pytest.approx(log2_tile), (w, n)


def test_fit_is_a_quadratic_in_log10_n():
    """Three or more points: the least-squares quadratic; the residual at
    the tuned points is the quadratic's, checked against numpy's own."""
    import numpy as np
    for w in (4, 8):
        pts = cf.table_points(cf.TABLES[w])
        coefs, _ = cf.fit(pts)
        x = np.array([p[0] for p in pts])
        y = np.array([p[1] for p in pts])
        ref = np.polyfit(x, y, min(2, len(pts) - 1))[::-1]
        assert np.allclose(coefs[:len(ref)], ref)


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


@pytest.mark.parametrize("dtype,w", [(torch.int32, 4), (torch.int64, 8)], ids=["int32", "int64"])
def test_library_default_follows_the_fit(evo, dtype, w):
    coefs, rng = cf.fits_from_tables()[w]
    for n in (1 << 20, 3 << 20, 1 << 22, 1 << 24, 1 << 26, 3 << 26, 1 << 28, 10 ** 9, 10 ** 10):
        want = cf.nearest_shape(w, cf.evaluate(coefs, rng, n))
        got = evo.resolve(n, dtype, algo="radix")
        assert (got["block_size"], got["keys_per_thread"]) == want, (n, got)
        assert got["pass_kernel"] == 2 and got["digit_bits"] == 8 and got["rank_mode"] == 4


def test_small_inputs_keep_the_fill_rule(evo):
    """Below the fitted range the default still gives half of the SMs a
    tile: a 1e5-key sort takes a tile far smaller than the fitted one."""
    got = evo.resolve(100_000, torch.int32, algo="radix")
    assert got["block_size"] * got["keys_per_thread"] < 8192
    # an explicit shape is kept as given
    got = evo.resolve(10 ** 9, torch.int32, algo="radix", block_size=512, keys_per_thread=16)
    assert (got["block_size"], got["keys_per_thread"]) == (512, 16)
