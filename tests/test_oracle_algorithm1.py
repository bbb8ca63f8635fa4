"""Pins of the order of Algorithm 1's base-layer search (bracketing, then bisection).

The end-to-end invariants (every point within the bound, the fallback never
longer than base-only, determinism) hold whatever ratio the search settles on,
so they cannot tell a swapped branch, an e_f taken from the wrong evaluation or
a missing reset of q_A from the printed algorithm.  Here the oracle's own loop
runs against hand-made q_A(r) curves instead of the JPEG 2000 encoder, and the
sequence of evaluated ratios and the evaluation kept as e_f are compared with
traces worked out by hand from Algorithm 1 (Materials and Methods).  The loop
halves r_low while q_A < q, keeps the last encoding as e_f, resets q_A to q_A0,
doubles r_high while q_A > q, then bisects while r_high - r_low > tol: a
midpoint with q_A < q becomes r_high, any other becomes r_low and e_f.  The
readings pinned with it: r_low floored at 1 (c14), r_high capped at r_max, and
the q = 1 fallback doubling while q_A >= q (c17).

Every case uses r0 = 20 and, unless stated, q = 0.999 and tol = 2.5 so that
each trace is short enough to derive by hand.
"""
import oracle as O

Q = 0.999
TOL = 2.5


def step(*feasible_intervals):
    """q_A(r) = 1 on the given closed intervals of r, 0.5 elsewhere."""
    def qa(r):
        return 1.0 if any(a <= r <= b for a, b in feasible_intervals) else 0.5
    return qa


def test_feasible_at_r0():
    """q_A = 1 for r <= 30.
    r0 = 20 meets q: no halving, e_f = e(20).  q_A0 = 1 > q: double to 40,
    which misses q, so the bracket is [20, 40].  Bisection: 30 meets q ->
    r_low = 30, e_f = e(30) (width 10); 35 misses -> r_high = 35 (width 5);
    32.5 misses -> r_high = 32.5 (width 2.5, not above tol: stop)."""
    seq, kept, r_f, q_f, ok = O.base_loop_trace(step((0, 30)), r0=20, tol=TOL, q=Q)
    assert seq == [20, 40, 30, 35, 32.5]
    assert kept == 2 and r_f == 30 and q_f == 1.0 and ok


def test_infeasible_at_r0():
    """q_A = 1 for r <= 7.
    20 misses -> halve: 10 misses -> halve: 5 meets q, stop; e_f = e(5).
    q_A is reset to q_A0 = 0.5, which is not above q: no doubling, r_high
    stays 20.  Bisection of [5, 20]: 12.5 misses -> r_high (width 7.5);
    8.75 misses -> r_high (width 3.75); 6.875 meets q -> r_low, e_f
    (width 1.875: stop)."""
    seq, kept, r_f, q_f, ok = O.base_loop_trace(step((0, 7)), r0=20, tol=TOL, q=Q)
    assert seq == [20, 10, 5, 12.5, 8.75, 6.875]
    assert kept == 5 and r_f == 6.875 and ok


def test_e_f_from_the_halving_loop():
    """q_A = 1 for r <= 5.
    20, 10 miss; 5 meets q: e_f = e(5).  No doubling (q_A0 misses).  The
    bisection of [5, 20] meets q nowhere (12.5, 8.75, 6.875 all miss), so e_f
    stays the encoding made at r_low = 5 by the halving loop."""
    seq, kept, r_f, q_f, ok = O.base_loop_trace(step((0, 5)), r0=20, tol=TOL, q=Q)
    assert seq == [20, 10, 5, 12.5, 8.75, 6.875]
    assert kept == 2 and r_f == 5 and ok


def test_non_monotone_curve_keeps_r_low_at_r0_while_doubling():
    """q_A = 1 for r <= 24 and for 36 <= r <= 45.
    20 meets q.  Doubling: 40 meets q (r_low stays at r0 = 20, as printed),
    80 misses: bracket [20, 80].  Bisection: 50 misses -> r_high (width 30);
    35 misses -> r_high (15); 27.5 misses -> r_high (7.5); 23.75 meets q ->
    r_low, e_f (3.75); 25.625 misses -> r_high (1.875: stop)."""
    seq, kept, r_f, q_f, ok = O.base_loop_trace(step((0, 24), (36, 45)), r0=20, tol=TOL, q=Q)
    assert seq == [20, 40, 80, 50, 35, 27.5, 23.75, 25.625]
    assert kept == 6 and r_f == 23.75 and ok


def test_no_ratio_feasible_floors_at_one():
    """q_A = 0.5 everywhere.  Halving 20, 10, 5, 2.5, 1.25, then 0.625 is
    floored to 1, after which the halving stops (r_low <= 1); e_f = e(1).
    No doubling.  Bisection of [1, 20]: 10.5 (width 9.5), 5.75 (4.75), 3.375
    (2.375: stop), all missing q.  The kept encoding misses q."""
    seq, kept, r_f, q_f, ok = O.base_loop_trace(step(), r0=20, tol=TOL, q=Q)
    assert seq == [20, 10, 5, 2.5, 1.25, 1.0, 10.5, 5.75, 3.375]
    assert kept == 5 and r_f == 1.0 and q_f == 0.5 and not ok


def test_doubling_capped_at_r_max():
    """q_A = 1 everywhere, r_max = 100.  Doubling 40, 80; 160 would pass
    r_max: stop.  Bisection of [20, 80]: 50, 65, 72.5, 76.25, 78.125 all meet
    q (widths 30, 15, 7.5, 3.75, 1.875), each becoming r_low and e_f."""
    seq, kept, r_f, q_f, ok = O.base_loop_trace(step((0, 1e9)), r0=20, tol=TOL, q=Q, r_max=100)
    assert seq == [20, 40, 80, 50, 65, 72.5, 76.25, 78.125]
    assert kept == 7 and r_f == 78.125 and ok


def test_q1_fallback_upward_condition():
    """q = 1, q_A = 1 for r <= 30 and 0.9999 above.  With the fallback's
    reading (c17: double while q_A >= q) the trace is that of
    test_feasible_at_r0.  With the printed test q_A > q the doubling can never
    start at q = 1, the bracket is [20, 20] and only r0 is evaluated."""
    def qa(r):
        return 1.0 if r <= 30 else 0.9999
    seq, kept, r_f, _, ok = O.base_loop_trace(qa, r0=20, tol=TOL, q=1.0, fallback=True)
    assert seq == [20, 40, 30, 35, 32.5] and kept == 2 and r_f == 30 and ok
    seq, kept, r_f, _, ok = O.base_loop_trace(qa, r0=20, tol=TOL, q=1.0, fallback=False)
    assert seq == [20] and kept == 0 and r_f == 20 and ok


def test_default_tolerance_step_count():
    """With the printed tol = 1e-3 and q_A = 1 for r <= 30: r0 = 20, doubling
    to 40, then bisection of a width-20 bracket until the width is at most
    1e-3: 20 / 2^15 = 6.1e-4 is the first, so 15 midpoints.  The first (30)
    meets q; every later one, 30 + 10 / 2^k, misses, so r_f = 30."""
    seq, kept, r_f, _, ok = O.base_loop_trace(step((0, 30)), r0=20, tol=1e-3, q=Q)
    assert len(seq) == 2 + 15
    assert seq[2] == 30 and all(seq[2 + k] == 30 + 10 / 2 ** k for k in range(1, 15))
    assert kept == 2 and r_f == 30 and ok
