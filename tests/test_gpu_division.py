"""The merge divides on the integer units when it computes the exact
centres of Eq. 4 (four correctly rounded binary64 divisions per local group).
jabba_check_division runs that path beside the GPU's own binary64 division
on the same operands and counts the quotients that differ in any bit: random
operands over a wide exponent range, exact quotients (zero remainder; a
quotient of two 53-bit significands is never halfway between two doubles),
power-of-two divisors, operands on either side of the significand
comparison, and the member-count divisors 1..4096 through their table."""
import numpy as np
import pytest

from _gpu import ctx

pytestmark = pytest.mark.gpu


def _dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


def _random_operands(rng, n):
    a = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-300, 300, n)) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-300, 300, n))
    return a, b


def test_random_quotients_match_binary64():
    C = ctx()
    rng = np.random.default_rng(11)
    a, b = _random_operands(rng, 1 << 22)
    handled, bad = C.check_division(_dev(a), _dev(b), mode=0)
    assert bad == 0
    assert handled == a.size  # every operand and quotient here is normal


def test_exact_quotients_powers_of_two_and_significand_order():
    C = ctx()
    rng = np.random.default_rng(12)
    n = 1 << 20
    # exact quotients: a = q b with q b below 2^53 (zero remainder)
    b_ex = (2 * rng.integers(0, 1 << 20, n) + 1).astype(np.float64)
    q_ex = rng.integers(1, 1 << 32, n).astype(np.float64)
    a_ex = q_ex * b_ex * np.exp2(rng.integers(-40, 40, n))
    # power-of-two divisors (the table's largest reciprocal) and equal significands
    a_p2, _ = _random_operands(rng, n)
    b_p2 = np.exp2(rng.integers(-200, 200, n)).astype(np.float64)
    a_eq = rng.uniform(1.0, 2.0, n)
    b_eq = a_eq * np.exp2(rng.integers(-5, 5, n))
    # significands one unit apart either way, and small odd divisors
    a_nb = rng.uniform(1.0, 2.0, n)
    b_nb = np.nextafter(a_nb, np.where(rng.random(n) < 0.5, 0.0, 4.0))
    a_odd = rng.integers(1, 1 << 53, n).astype(np.float64)
    b_odd = (2 * rng.integers(0, 50, n) + 1).astype(np.float64)
    for a, b in [(a_ex, b_ex), (a_p2, b_p2), (a_eq, b_eq), (a_nb, b_nb), (a_odd, b_odd)]:
        handled, bad = C.check_division(_dev(a), _dev(b), mode=0)
        assert bad == 0
        assert handled == a.size
    # zeros of either sign: +-0 / b keeps the sign
    z = np.array([0.0, -0.0, 0.0], np.float64)
    handled, bad = C.check_division(_dev(z), _dev(np.array([3.0, 7.0, 1.0])), mode=0)
    assert (handled, bad) == (3, 0)


def test_member_count_divisors_through_the_table():
    C = ctx()
    rng = np.random.default_rng(13)
    counts = np.tile(np.arange(1, 4097, dtype=np.float64), 512)
    # length sums (integers below 2^24) and increment sums (any sign and scale)
    lensum = (counts * rng.uniform(1.0, 4096.0, counts.size)).round().clip(1, None)
    inc, _ = _random_operands(rng, counts.size)
    for a in (lensum, inc):
        handled, bad = C.check_division(_dev(a), _dev(counts), mode=1)
        assert bad == 0
        assert handled == counts.size
    # values that are not counts are skipped
    handled, bad = C.check_division(_dev(np.ones(4)), _dev(np.array([0.0, 4097.0, 2.5, -3.0])), mode=1)
    assert (handled, bad) == (0, 0)
