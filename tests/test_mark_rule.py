"""The resident engine's narrowed dirty marks, checked on the CPU.

The engine re-tests a point only if some neighbour moved since its last test,
and of a moved neighbour p (lowered from c0 to c1 in its phase) it marks only
the neighbours q with c1 < F(q) <= c0 + lambda (saturated).  The claim: the
test of Sec. 2.1 sees p only through "p < F(q)" and "p < F(q) - lambda", and
the lowering loop of Sec. 2.2 skips every neighbour value strictly between
two of its steps, so for every other q neither bit changes and neither does
q's test result.  Thinning with dirty sets under that rule must then give
exactly the image, lowering count and last changing phase of the plain
subfield schedule (the oracle).  Small images with few grey levels put many
equal values side by side, where an off-by-one in the rule would show.  A
rule that drops the equal values (c1 < F(q) < c0 + lambda) must fail on the
same cases: the test can tell a wrong rule from the right one."""
import numpy as np
import pytest

import oracle

RING = [(1, 0), (1, -1), (0, -1), (-1, -1), (-1, 0), (-1, 1), (0, 1), (1, 1)]  # E, NE, N, NW, W, SW, S, SE


def thin_dirty(img, lam, rule, op, adj, upper_inclusive=True, cap=True):
    """Subfield schedule (phase g visits parity g mod 4 in raster order) that tests only dirty points.
    cap=False drops the upper bound (the engine's wide mode marks every neighbour above c1)."""
    F = img.astype(np.int64).copy()
    h, w = F.shape
    dirty = np.ones((h, w), bool)
    lowered, last, g = 0, -1, 0
    while True:
        round_changed = False
        for _ in range(4):
            p = g % 4
            changed = False
            for y in range(1, h - 1):
                if (y & 1) != (p >> 1):
                    continue
                for x in range(1, w - 1):
                    if (x & 1) != (p & 1) or not dirty[y, x]:
                        continue
                    dirty[y, x] = False
                    nb = [int(F[y + dy, x + dx]) for dx, dy in RING]
                    c0 = int(F[y, x])
                    while True:
                        ok, alpha = oracle.lowerable(nb, int(F[y, x]), lam, rule, op, adj)
                        if not ok:
                            break
                        F[y, x] = alpha
                        lowered += 1
                    c1 = int(F[y, x])
                    if c1 == c0:
                        continue
                    changed = True
                    hi = min(c0 + lam, 1 << 30) if cap else 1 << 30
                    for (dx, dy), v in zip(RING, nb):
                        qx, qy = x + dx, y + dy
                        if not (1 <= qx < w - 1 and 1 <= qy < h - 1):
                            continue
                        if c1 < v and (v <= hi if upper_inclusive else v < hi):
                            dirty[qy, qx] = True
            if changed:
                round_changed = True
                last = g
            g += 1
        if not round_changed:
            break
    return F.astype(img.dtype), lowered, last


CASES = [(seed, lam, rule, op, adj)
         for seed in (1, 2)
         for lam in (0, 1, 3)
         for (rule, op, adj) in ((oracle.RULE_MAX, oracle.OP_THIN, oracle.ADJ_8_4),
                                 (oracle.RULE_MIN, oracle.OP_THIN, oracle.ADJ_8_4),
                                 (oracle.RULE_MAX, oracle.OP_SKELETON, oracle.ADJ_8_4),
                                 (oracle.RULE_MAX, oracle.OP_THIN, oracle.ADJ_4_8))]


def image(seed):
    rng = np.random.default_rng(seed)
    # few grey levels, smooth enough to leave plateaus and ridges: many equal neighbours
    a = rng.integers(0, 6, size=(9, 11)).astype(np.float64)
    a = np.kron(a, np.ones((2, 2)))[:17, :21] + rng.integers(0, 2, size=(17, 21))
    return a.astype(np.uint8)


@pytest.mark.parametrize("cap", [True, False])
@pytest.mark.parametrize("seed,lam,rule,op,adj", CASES)
def test_narrow_marks_give_the_oracle_result(seed, lam, rule, op, adj, cap):
    img = image(seed)
    ref, st = oracle.thin(img, lam, rule=rule, op=op, adj=adj)
    out, lowered, last = thin_dirty(img, lam, rule, op, adj, cap=cap)
    assert np.array_equal(out, ref)
    assert lowered == st["lowered"] and last == st["last_change_phase"]


def test_a_rule_that_drops_equal_values_is_caught():
    wrong = 0
    for seed, lam, rule, op, adj in CASES:
        img = image(seed)
        ref, st = oracle.thin(img, lam, rule=rule, op=op, adj=adj)
        out, lowered, _ = thin_dirty(img, lam, rule, op, adj, upper_inclusive=False)
        wrong += int(not np.array_equal(out, ref) or lowered != st["lowered"])
    assert wrong > 0
