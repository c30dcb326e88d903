"""The inter-sweep schedule of the band -> tridiagonal bulge chasing, checked on the host.

A model of which entries (row, column) of the lower band each phase of each step reads and writes:
step k of sweep s (r0 = s+1+kb, L = min(b, n-r0), c = s for k = 0, else s+1+(k-1)b):

  A  k = 0: reads and rewrites column c, rows r0 .. r0+L-1 (the annihilated column);
     k > 0: stores the row block rows r0 .. r0+L-1 x columns c .. c+b-1, which the previous step's
     phase C read from the band and kept;
  B  reads and rewrites the lower triangle of the diagonal block rows/columns r0 .. r0+L-1;
  C  reads the block below, rows r0+L .. r0+L+L2-1 x columns r0 .. r0+L-1 (L2 = min(b, n-r0-L)),
     writing it back only at the last step of the sweep (otherwise the next step's A stores it).

Progress of a sweep counts half steps: 2j+1 after A of step j, 2j+2 after step j.  A sweep starts
step k once the previous sweep's progress reaches `need(k)`.  A schedule is safe when nothing a
step reads or writes is written, or held stale, by a still-pending operation of the sweeps ahead,
and nothing it writes is read by one; the sweep two ahead is checked at the least progress the
rule allows it.  The half-step rule of the kernel (2(k+2)+1) and the whole-step rule (2(k+3)) must
be safe; the rule one half step weaker than the kernel's (2(k+2)) must not be.
"""
import pytest


def sweep_steps(n, b, s):
    """Steps of sweep s: windows r0 = s+1+kb with at least two rows (min(b, n - r0) >= 2)."""
    if s > n - 3:
        return 0
    return (n - s - 3) // b + 1


def step_sets(n, b, s, k):
    """(reads, writes) of phases A, B, C of step k of sweep s, as sets of (row, column)."""
    nst = sweep_steps(n, b, s)
    r0 = s + 1 + k * b
    L = min(b, n - r0)
    c = s if k == 0 else s + 1 + (k - 1) * b
    A = set()
    if k == 0:
        A = {(r0 + i, c) for i in range(L)}
    else:
        A = {(r0 + i, c + cc) for i in range(L) for cc in range(b)}
    B = {(r0 + i, r0 + j) for i in range(L) for j in range(L) if i >= j}
    rn0 = r0 + L
    L2 = min(b, n - rn0)
    C = {(rn0 + i, r0 + j) for i in range(max(L2, 0)) for j in range(L)}
    last = (k + 1 == nst)
    return {"A": (A, A), "B": (B, B), "C": (C, C if last else set())}


def pending(n, b, s, P):
    """Reads and writes of sweep s still to come at progress P (half steps)."""
    pr, pw = set(), set()
    for j in range(sweep_steps(n, b, s)):
        ph = step_sets(n, b, s, j)
        if P <= 2 * j:                 # A of step j not done: its store (and reads) are pending
            pr |= ph["A"][0]
            pw |= ph["A"][1]
        if P <= 2 * j + 1:             # B and C of step j not done
            for key in ("B", "C"):
                pr |= ph[key][0]
                pw |= ph[key][1]
    return pr, pw


def check(n, b, need):
    """True when every step of every sweep is safe against the two sweeps ahead of it."""
    for s in range(1, max(n - 2, 1)):
        for k in range(sweep_steps(n, b, s)):
            P1 = need(k, sweep_steps(n, b, s - 1))
            ph = step_sets(n, b, s, k)
            touch = set().union(*(ph[x][0] | ph[x][1] for x in "ABC"))
            writes = set().union(*(ph[x][1] for x in "ABC"))
            pr, pw = pending(n, b, s - 1, P1)
            if touch & pw or writes & pr:
                return False
            if s >= 2 and P1 < 2 * sweep_steps(n, b, s - 1):
                # sweep s-1 is inside step P1 // 2; its start needed sweep s-2 at need(P1 // 2)
                P2 = need(P1 // 2, sweep_steps(n, b, s - 2))
                pr2, pw2 = pending(n, b, s - 2, P2)
                if touch & pw2 or writes & pr2:
                    return False
    return True


def half_rule(k, prev_nst):
    return min(2 * k + 5, 2 * prev_nst)


def whole_rule(k, prev_nst):
    return min(2 * k + 6, 2 * prev_nst)


def too_weak(k, prev_nst):
    return min(2 * k + 4, 2 * prev_nst)


SHAPES = [(12, 2), (23, 3), (40, 4), (41, 5), (57, 8), (70, 4), (33, 16)]


@pytest.mark.parametrize("n,b", SHAPES)
def test_half_step_rule_is_safe(n, b):
    assert check(n, b, half_rule)


@pytest.mark.parametrize("n,b", SHAPES)
def test_whole_step_rule_is_safe(n, b):
    assert check(n, b, whole_rule)


@pytest.mark.parametrize("n,b", [(23, 3), (40, 4), (57, 8)])
def test_one_half_step_less_conflicts(n, b):
    """Step k+2's row-block store must precede the next sweep's step k: without it they collide
    on one entry (row s+(k+2)b, column s+(k+1)b in the next sweep's indexing)."""
    assert not check(n, b, too_weak)
