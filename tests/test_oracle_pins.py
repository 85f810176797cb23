"""The CPU oracle pinned to closed forms, brute force, library routines and
invariants (no GPU).  See ``tests/pins.py`` for the individual pins."""
import pytest

import oracle
from tests import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", pins.PINS, ids=lambda f: f.__name__)
def test_pin(lib, pin):
    assert pin(lib)


def test_fig2_delegate_numbering(lib):
    """Fig. 2 / Sec. III-B: with TH=5, vertices 7 and 8 become delegates 0 and 1."""
    from tests.golden_io import read_fig2

    th, n, delegates, src, dst = read_fig2()
    g = oracle.Graph(n, src, dst, lib=lib)
    io, co, d, n_ni = g.separate(th)
    assert d == len(delegates)
    for v, want in delegates.items():
        assert io[v] == want and co[want] == v
    deg = g.degree()
    assert ((deg > th) == (io < d)).all()
