"""The data-movement ordering of the FP32 refinement Jacobi (host-side model).

The sweeps keep pair P of every step at positions (2P, 2P+1) and move every
matrix element from (x, y) to (pi(x), pi(y)) after each step.  The kernel
relies on four facts about that seat rotation, checked here for every even
n up to 128 on a plain model of it:

* pi is a permutation of the positions;
* the players at (2P, 2P+1) in step t are the round-robin pair of the
  one-CTA kernel, (n-1, t) for P = 0 and ((t+P) mod (n-1), (t-P) mod (n-1))
  otherwise (the closed form jacobi_vapply_kernel uses);
* every unordered pair of players meets exactly once in n-1 steps;
* after n-1 steps every player is back at its first position (the kernel
  reads the eigenvalues there).
"""
import itertools

import pytest


def seat_rotation(x, n):
    """pi: position 0 stays, first members move down one pair, second up."""
    if n == 2 or x == 0:
        return x
    if x == 2:
        return 1
    if x % 2 == 0:
        return x - 2
    if x == n - 1:
        return n - 2
    return x + 2


def first_seating(x, n):
    if x == 0:
        return n - 1
    if x == 1:
        return 0
    return n - 1 - x // 2 if x % 2 else x // 2


def closed_form_pair(t, P, n):
    if P == 0:
        return n - 1, t
    return (t + P) % (n - 1), (t - P) % (n - 1)


@pytest.mark.parametrize("n", list(range(2, 129, 2)))
def test_seat_rotation_schedule(n):
    np_ = n // 2
    assert sorted(seat_rotation(x, n) for x in range(n)) == list(range(n))
    seat = [first_seating(x, n) for x in range(n)]
    assert sorted(seat) == list(range(n))
    met = set()
    for t in range(n - 1):
        for P in range(np_):
            pair = (seat[2 * P], seat[2 * P + 1])
            assert pair == closed_form_pair(t, P, n), (t, P)
            met.add(frozenset(pair))
        moved = [0] * n
        for x in range(n):
            moved[seat_rotation(x, n)] = seat[x]
        seat = moved
    assert len(met) == n * (n - 1) // 2
    assert met == {frozenset(p) for p in itertools.combinations(range(n), 2)}
    assert seat == [first_seating(x, n) for x in range(n)]
