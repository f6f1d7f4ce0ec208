"""Host check of the block-step indexing (no GPU).

In a shared-memory step on digits J .. J+DD-1 of the HL row digits a CTA holds
(Algorithm 3, Section 4.1, several digits per step), work item r (one per
thread, strided over the CTA) takes the block of 3^DD rows base + t * 3^J,
t < 3^DD:
* Merge: base = lo + 3^(J+DD) * spread3(hb), lo < 3^J any, hb < 2^(HL-J-DD)
  spread to base-3 digits 0/1 (the digits above the step not merged yet must
  be 0/1);
* Reduce: base = lo + 3^(J+DD) * hi, lo < 3^J, hi < 3^(HL-J-DD).
The blocks of one step must be disjoint (the step works in place and one
barrier ends it), stay inside the 3^HL rows, and cover exactly the rows the
step must touch.  Checked for every shape the kernels instantiate: HL = 7
starting at the inner digits (streaming passes) and HL = 1..9 from digit 0
(whole functions), two and three digits per step.
"""
import pytest


def pow3(k):
    return 3 ** k


def spread3(x, k):
    return sum(pow3(i) for i in range(k) if (x >> i) & 1)


def digits_of(r, k):
    return [(r // pow3(i)) % 3 for i in range(k)]


def steps(HL, J0, D):
    J = J0
    while J < HL:
        DD = min(D, HL - J)
        yield J, DD
        J += DD


def merge_blocks(HL, J, DD):
    P, T = pow3(J), pow3(DD)
    for r in range(P * (1 << (HL - J - DD))):
        lo, hb = r % P, r // P
        base = lo + pow3(J + DD) * spread3(hb, HL - J - DD)
        yield [base + t * P for t in range(T)]


def reduce_blocks(HL, J, DD):
    P, T = pow3(J), pow3(DD)
    for r in range(pow3(HL - DD)):
        lo, hi = r % P, r // P
        base = lo + hi * pow3(J + DD)
        yield [base + t * P for t in range(T)]


SHAPES = [(7, b, d) for b in range(0, 7) for d in (2, 3)] + \
         [(hl, 0, d) for hl in range(1, 10) for d in (2, 3)]


@pytest.mark.parametrize("HL,J0,D", SHAPES)
def test_blocks_disjoint_in_bounds_and_covering(HL, J0, D):
    N = pow3(HL)
    for J, DD in steps(HL, J0, D):
        seen = set()
        for block in merge_blocks(HL, J, DD):
            assert all(0 <= x < N for x in block)
            assert not seen.intersection(block)
            seen.update(block)
        want = {x for x in range(N) if all(dg != 2 for dg in digits_of(x, HL)[J + DD:])}
        assert seen == want, ("merge", HL, J, DD)
        seen = set()
        for block in reduce_blocks(HL, J, DD):
            assert all(0 <= x < N for x in block)
            assert not seen.intersection(block)
            seen.update(block)
        assert seen == set(range(N)), ("reduce", HL, J, DD)


@pytest.mark.parametrize("HL,J0,D", SHAPES)
def test_block_rows_differ_only_in_the_step_digits(HL, J0, D):
    """Row t of a block has the step digits of t and the block's other digits."""
    for J, DD in steps(HL, J0, D):
        for blocks in (merge_blocks(HL, J, DD), reduce_blocks(HL, J, DD)):
            for block in blocks:
                d0 = digits_of(block[0], HL)
                assert d0[J:J + DD] == [0] * DD
                for t, x in enumerate(block):
                    d = digits_of(x, HL)
                    assert d[:J] == d0[:J] and d[J + DD:] == d0[J + DD:]
                    assert d[J:J + DD] == digits_of(t, DD)
