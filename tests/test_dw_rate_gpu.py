"""GPU test of fkk_dw_rate, the measured rate of the double-word multiply-add
that the eigensolver's tridiagonal reduction is made of.  The chains it
times must compute a <- a y + x_c in double-word arithmetic: thread 0's
values are compared with the same recurrence in exact rational arithmetic.

Tolerance: the sloppy double-word sum has an absolute error below
3 u^2 (|a y| + |x|) (u = 2^-24) and the product about 5 u^2 |a y|, about
1e-12 of a per step here; the recurrence contracts by y ~ 1 - 2^-9, so after
300 steps the error is below 300 * 1e-12 * a, rtol 1e-11 with margin.
Dropping the low word of y moves the result by ~1e-7 relative, and of x by
~1e-8, so both words are pinned."""
from fractions import Fraction

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2005_07132_gb300 import build
    build.build()
    import paper_2005_07132_gb300 as fk
    c = fk.Context(0)
    yield c
    c.close()


def _exact_chains(iters):
    f32 = lambda v: Fraction(float(torch.tensor(v, dtype=torch.float32)))  # noqa: E731
    y = (1 - Fraction(1, 2**9)) + 3 * Fraction(1, 2**33)
    x0 = f32(0.1) + Fraction(1, 2**30)
    out = []
    for c in range(8):
        x = x0 / 2**c
        a = Fraction(0)
        for _ in range(iters):
            a = a * y + x
        out.append(a)
    return out


def test_dw_rate_chains_are_double_word_exact(ctx):
    rate, chains = ctx.dw_rate(300)
    want = _exact_chains(300)
    for got, w in zip(chains, want):
        assert abs(Fraction(got) - w) <= Fraction(1, 10**11) * abs(w), (got, float(w))
    assert rate > 0.0


def test_dw_rate_is_plausible(ctx):
    rate, _ = ctx.dw_rate(4096)
    # fp32 lanes x clock / ~20 instructions per multiply-add, two flops: a few
    # 1e12 double-word flop/s on this part; the bounds only catch a broken timer
    assert 1e11 < rate < 4e13, rate


def test_dw_rate_rejects_bad_arguments(ctx):
    from paper_2005_07132_gb300 import FkkError
    with pytest.raises(FkkError):
        ctx.dw_rate(0)
