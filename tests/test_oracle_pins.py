"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: the references are hand-worked
cases (tests/golden), a textbook identity of (8,4) digital topology, global
component counts by scipy labelling (brute force), closed forms of the lambda
rule, and invariants of the operator (Sec. 2.1-2.2).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1603_09180_gb300.synth import uniform_noise_image, value_noise_image
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "point_cases.json")
RULES = {"max": oracle.RULE_MAX, "min": oracle.RULE_MIN}


def lower_mask(grid):
    g = np.asarray(grid)
    nb = bf.ring_values(g)
    return sum(1 << i for i, v in enumerate(nb) if v < g[1, 1])


# ---------------------------------------------------------------- point test

def test_golden_point_cases():
    cases = json.load(open(GOLDEN))["cases"]
    assert len(cases) >= 8
    for c in cases:
        g = np.array(c["grid"])
        tp, tm, _ = oracle.mask_numbers(lower_mask(g))
        assert (tp, tm) == (c["tplus"], c["tminus"]), c["name"]
        assert (tp == 1 and tm == 1) == c["destructible"], c["name"]
        for chk in c["checks"]:
            ok, alpha = oracle.lambda_destructible(bf.ring_values(g), g[1, 1], chk["lam"], RULES[chk["rule"]])
            assert ok == chk["first"], (c["name"], chk)
            if ok:
                assert alpha == c["alpha"], c["name"]
            out, st = oracle.thin(g.astype(np.int32), chk["lam"], RULES[chk["rule"]])
            assert out[1, 1] == chk["final"], (c["name"], chk)
            # the border of a 3x3 image is never written
            mask = np.ones((3, 3), bool)
            mask[1, 1] = False
            assert (out[mask] == g[mask]).all()


def test_84_identity_all_masks():
    """(8,4) in 2-D: T+ = T-- except at a 4-interior point (no strictly lower
    4-neighbour, lower corners allowed: T+ = 1, T-- = 0) and an isolated point
    (all eight lower: T+ = 0, T-- = 1)."""
    four = 0b01010101  # E, N, W, S
    for m in range(256):
        tp, tm, _ = oracle.mask_numbers(m)
        if m & four == 0:
            assert (tp, tm) == (1, 0)
        elif m == 255:
            assert (tp, tm) == (0, 1)
        else:
            assert tp == tm, m
        assert 0 <= tp <= 4 and 0 <= tm <= 4


def test_all_masks_against_scipy_labelling():
    for m in range(256):
        nb = [0 if (m >> i) & 1 else 2 for i in range(8)]
        g = bf.grid_from_ring(1, nb)
        tp_ref, tm_ref, comps = bf.local_numbers(g)
        tp, tm, lab = oracle.mask_numbers(m)
        assert (tp, tm) == (tp_ref, tm_ref), m
        # same partition of the lower neighbours into counted components
        ref_part = {frozenset(c) for c in comps}
        got = {}
        for i, l in enumerate(lab):
            if l >= 0:
                got.setdefault(l, set()).add(bf.RING_RC[i])
        assert {frozenset(s) for s in got.values()} == ref_part, m


def test_tplusplus_matches_labelling():
    for m in range(256):
        g = bf.grid_from_ring(1, [2 if (m >> i) & 1 else 1 for i in range(8)])
        up = g > 1
        up[1, 1] = False
        assert oracle.tplusplus(m) == bf.components(up, bf.EIGHT)


def test_simple_count_among_masks():
    """Number of ring configurations with T+ = 1 and T-- = 1 (simple points of
    a binary set under (8,4)), cross-checked against the global brute force."""
    simple = [m for m in range(256) if oracle.mask_numbers(m)[:2] == (1, 1)]
    glob = []
    for m in range(256):
        img = np.full((5, 5), 1, dtype=np.int32)
        g = bf.grid_from_ring(1, [0 if (m >> i) & 1 else 1 for i in range(8)])
        img[1:4, 1:4] = g
        # outer ring at 1: the lower neighbours (0) only touch each other through x
        if bf.global_destructible(img, 2, 2) and m != 0:
            glob.append(m)
    assert simple == glob


@pytest.mark.parametrize("outer", ["zeros", "ones", "twos", "random"])
def test_local_equals_global_all_masks(outer):
    rng = np.random.default_rng(5)
    for m in range(256):
        img = {"zeros": np.zeros((5, 5)), "ones": np.ones((5, 5)), "twos": np.full((5, 5), 2),
               "random": rng.integers(0, 3, (5, 5))}[outer].astype(np.int32)
        img[1:4, 1:4] = bf.grid_from_ring(1, [0 if (m >> i) & 1 else 2 for i in range(8)])
        local, _ = oracle.lambda_destructible(bf.ring_values(img[1:4, 1:4]), 1, 0)
        assert local == oracle.global_destructible(img, 2, 2) == bf.global_destructible(img, 2, 2), (m, outer)


@pytest.mark.parametrize("shape,levels,count", [((4, 4), 3, 3000), ((5, 5), 3, 1500), ((8, 8), 4, 150)])
def test_local_equals_global_random_images(shape, levels, count):
    rng = np.random.default_rng(11 + shape[0])
    h, w = shape
    for _ in range(count):
        img = rng.integers(0, levels, shape).astype(np.int32)
        for y in range(1, h - 1):
            for x in range(1, w - 1):
                local, _ = oracle.lambda_destructible(bf.ring_values(img[y - 1:y + 2, x - 1:x + 2]), img[y, x], 0)
                assert local == oracle.global_destructible(img, x, y), (img, x, y)
                if count <= 150:
                    assert local == bf.global_destructible(img, x, y)


def test_lambda_rule_against_reference():
    rng = np.random.default_rng(3)
    for _ in range(4000):
        g = rng.integers(0, 7, (3, 3))
        nb = bf.ring_values(g)
        for lam in (0, 1, 2, 4):
            for rule in (0, 1):
                got = oracle.lambda_destructible(nb, g[1, 1], lam, rule)
                ref = bf.point_step(g, lam, rule)
                assert got[0] == ref[0], (g, lam, rule)
                if got[0]:
                    assert got[1] == ref[1]


def test_lambda_closed_forms():
    rng = np.random.default_rng(8)
    for _ in range(3000):
        g = rng.integers(0, 9, (3, 3))
        nb, c = bf.ring_values(g), int(g[1, 1])
        d0 = oracle.lambda_destructible(nb, c, 0)[0]
        tp, tm, _ = oracle.mask_numbers(lower_mask(g))
        # lambda = 0: components are strictly lower, so only destructible points qualify
        assert d0 == (tp == 1 and tm == 1)
        prev = d0
        for lam in range(1, 10):
            cur = oracle.lambda_destructible(nb, c, lam)[0]
            assert cur >= prev  # monotone in lambda
            prev = cur
        ok, alpha = oracle.lambda_destructible(nb, c, 9)
        if ok:
            assert alpha == max(v for v in nb if v < c) < c
        if tm >= 2 and prev:
            # a k-divergent point at lambda >= its full contrast is always lambda-destructible
            assert oracle.lambda_destructible(nb, c, c)[0]
        # constant-valued components: R1 and R2 agree
        if len({v for v in nb if v < c}) <= 1:
            for lam in range(0, 10):
                assert oracle.lambda_destructible(nb, c, lam, 0)[0] == oracle.lambda_destructible(nb, c, lam, 1)[0]


# ---------------------------------------------------------------- schedule

@pytest.mark.parametrize("lam,rule", [(0, 0), (1, 0), (3, 0), (2, 1)])
def test_schedule_against_python_reference(lam, rule):
    rng = np.random.default_rng(100 + lam + 10 * rule)
    for _ in range(12):
        h, w = int(rng.integers(3, 9)), int(rng.integers(3, 10))
        img = rng.integers(0, 5, (h, w)).astype(np.int32)
        out, st = oracle.thin(img, lam, rule)
        assert np.array_equal(out, bf.schedule(img, lam, rule)), img
        assert st["converged"] == 1


def test_schedule_lambda0_against_global_brute_force():
    """At lambda = 0 each lowering is decided by global component counts of the
    threshold sections: the local point test must lead to the same image."""
    rng = np.random.default_rng(21)
    for _ in range(10):
        h, w = int(rng.integers(4, 8)), int(rng.integers(4, 8))
        img = rng.integers(0, 4, (h, w)).astype(np.int32)
        out, _ = oracle.thin(img, 0)
        assert np.array_equal(out, bf.schedule(img, 0, use_global=True)), img


def test_binary_reduces_to_simple_point_thinning():
    """A {0,1} image at lambda = 0 is binary thinning by deletion of simple
    points in the subfield order; deletion decided by global counts."""
    rng = np.random.default_rng(4)
    blob = np.zeros((14, 14), np.int32)
    for _ in range(6):
        y, x, r = rng.integers(2, 12), rng.integers(2, 12), rng.integers(1, 4)
        yy, xx = np.mgrid[:14, :14]
        blob[(yy - y) ** 2 + (xx - x) ** 2 <= r * r] = 1
    blob[0, :] = blob[-1, :] = blob[:, 0] = blob[:, -1] = 0
    out, _ = oracle.thin(blob, 0)
    ref = bf.schedule(blob, 0, use_global=True)
    assert np.array_equal(out, ref)
    assert set(np.unique(out)) <= {0, 1}
    assert (out <= blob).all()


def _invariants(img, out, lam):
    assert out.shape == img.shape and out.dtype == img.dtype
    assert (out <= img).all()
    assert oracle.count_lambda_destructible(out, lam) == 0
    b = np.ones(img.shape, bool)
    b[1:-1, 1:-1] = False
    assert (out[b] == img[b]).all()


@pytest.mark.parametrize("lam", [0, 5, 20])
def test_invariants_on_generator_images(lam):
    img = value_noise_image(40, 56, "u8", seed=7)
    out, st = oracle.thin(img, lam)
    _invariants(img, out, lam)
    assert st["converged"] == 1 and st["lowered"] > 0
    if lam == 0:
        assert oracle.level_topology(img) == oracle.level_topology(out, levels=sorted(oracle.level_topology(img)))


@pytest.mark.parametrize("variant", ["queue", "minvalue"])
@pytest.mark.parametrize("lam", [0, 6])
def test_other_orders_same_invariants(variant, lam):
    img = value_noise_image(32, 48, "u8", seed=9)
    f = oracle.thin_queue if variant == "queue" else oracle.thin_minvalue
    out, n = f(img, lam)
    _invariants(img, out, lam)
    sched, _ = oracle.thin(img, lam)
    if lam == 0:
        levels = sorted(oracle.level_topology(img))
        assert oracle.level_topology(out, levels) == oracle.level_topology(sched, levels) == oracle.level_topology(img, levels)


def test_constant_image_and_peak_unchanged():
    c = np.full((9, 11), 77, np.uint8)
    out, st = oracle.thin(c, 30)
    assert np.array_equal(out, c) and st["lowered"] == 0 and st["rounds"] == 1
    assert st["last_change_phase"] == -1
    p = np.full((9, 9), 10, np.uint8)
    p[4, 4] = 200
    out, st = oracle.thin(p, 0)
    assert np.array_equal(out, p)


@pytest.mark.parametrize("d,lam", [(3, 2), (3, 3), (5, 4), (5, 5), (5, 9)])
def test_flat_basins_merge_iff_depth_le_lambda(d, lam):
    H = 10
    img = np.full((15, 21), H, np.int32)
    img[4:11, 3:10] = H - d   # basin 1
    img[4:11, 11:18] = H - d  # basin 2, column 10 is a 1-px ridge
    out, _ = oracle.thin(img, lam)
    n_low = bf.components(out < H, bf.FOUR)
    assert n_low == (1 if d <= lam else 2)
    for rule in (0, 1):  # constant basins: the F^- reading does not matter
        assert np.array_equal(oracle.thin(img, lam, rule)[0], out)


def test_resume_equals_uninterrupted():
    img = value_noise_image(33, 47, "u8", seed=3)
    full, st = oracle.thin(img, 5)
    for k in (1, 3, 4, 9, 22):
        part, s1 = oracle.thin(img, 5, max_phases=k)
        assert s1["capped"] and s1["end_phase"] == k
        rest, s2 = oracle.thin(part, 5, start_phase=k)
        assert np.array_equal(rest, full)
        assert s1["lowered"] + s2["lowered"] == st["lowered"]


def test_u16_and_tiny_shapes():
    img = uniform_noise_image(12, 13, "u16", seed=2, vmax=65535)
    out, _ = oracle.thin(img, 1000)
    _invariants(img, out, 1000)
    for shape in [(0, 0), (1, 5), (2, 2), (5, 2), (3, 3)]:
        a = np.arange(int(np.prod(shape)), dtype=np.uint8).reshape(shape)
        o, st = oracle.thin(a, 0) if a.size else (a, None)
        if a.size and min(shape) < 3:
            assert np.array_equal(o, a)


def test_oracle_leaves_inputs_untouched():
    """The wrapper works on a copy for every input dtype (int32 included)."""
    for dt in (np.int32, np.uint8, np.uint16):
        img = (np.arange(64).reshape(8, 8) * 7 % 23).astype(dt)
        keep = img.copy()
        oracle.thin(img, 3)
        oracle.thin_queue(img, 3)
        oracle.thin_minvalue(img, 3)
        assert np.array_equal(img, keep)


# ---------------------------------------------------------------- lambda-skeleton (Sec. 2.2)

SK = oracle.OP_SKELETON


def test_skeleton_point_against_reference():
    rng = np.random.default_rng(31)
    for _ in range(4000):
        g = rng.integers(0, 7, (3, 3))
        if rng.random() < 0.2:  # more end points: one neighbour at or above the centre
            g[:] = rng.integers(0, 3)
            g[1, 1] = 5
            r, c = bf.RING_RC[int(rng.integers(8))]
            g[r, c] = int(rng.integers(5, 7))
        nb = bf.ring_values(g)
        for lam in (0, 1, 2, 4, 6):
            for rule in (0, 1):
                got = oracle.lambda_skeleton_point(nb, g[1, 1], lam, rule)
                ref = bf.skeleton_step(g, lam, rule)
                assert got[0] == ref[0], (g, lam, rule)
                if got[0]:
                    assert got[1] == ref[1]


@pytest.mark.parametrize("lam,rule", [(0, 0), (1, 0), (3, 0), (2, 1)])
def test_skeleton_schedule_against_python_reference(lam, rule):
    rng = np.random.default_rng(200 + lam + 10 * rule)
    for _ in range(12):
        h, w = int(rng.integers(3, 9)), int(rng.integers(3, 10))
        img = rng.integers(0, 5, (h, w)).astype(np.int32)
        out, st = oracle.thin(img, lam, rule, op=SK)
        assert np.array_equal(out, bf.schedule(img, lam, rule, op=1)), img
        assert st["converged"] == 1


def test_skeleton_lambda0_against_global_brute_force():
    """At lambda = 0 the skeleton lowers destructible points that are not end
    points (Sec. 2.2, first sentence); destructibility by global counts."""
    rng = np.random.default_rng(22)
    for _ in range(10):
        h, w = int(rng.integers(4, 8)), int(rng.integers(4, 8))
        img = rng.integers(0, 4, (h, w)).astype(np.int32)
        out, _ = oracle.thin(img, 0, op=SK)
        assert np.array_equal(out, bf.schedule(img, 0, use_global=True, op=1)), img


@pytest.mark.parametrize("d,lam", [(40, 0), (40, 39), (40, 40), (40, 80)])
@pytest.mark.parametrize("diag", [False, True])
def test_skeleton_keeps_a_line_iff_its_contrast_exceeds_lambda(d, lam, diag):
    """A one-pixel line of contrast d on a flat background: every inner pixel
    is not simple and both ends are end points, so the skeleton keeps the line
    while d > lambda (its ends are lambda-end); once d <= lambda the ends are
    lambda-deletable and the line is eaten down to the background.  Plain
    lambda-thinning (d > lambda) erodes the line from its ends to a single
    peak pixel."""
    img = np.full((20, 20), 100, np.int32)
    for k in range(3, 16):
        if diag:
            img[k, k] = 100 + d
        else:
            img[9, k] = 100 + d
    out, _ = oracle.thin(img, lam, op=SK)
    if d > lam:
        assert np.array_equal(out, img)
    else:
        assert (out == 100).all()
    if d > lam:
        thin_out, _ = oracle.thin(img, lam)
        assert (thin_out == 100 + d).sum() == 1 and (thin_out > 100).sum() == 1


@pytest.mark.parametrize("d,lam", [(5, 4), (5, 5), (5, 9)])
def test_skeleton_removes_a_peak_iff_its_height_le_lambda(d, lam):
    img = np.full((9, 9), 50, np.int32)
    img[4, 4] = 50 + d
    out, _ = oracle.thin(img, lam, op=SK)
    assert out[4, 4] == (50 if d <= lam else 50 + d)
    assert oracle.thin(img, lam)[0][4, 4] == 50 + d  # a peak is never lambda-destructible


def _skeleton_invariants(img, out, lam):
    assert (out <= img).all()
    assert oracle.count_lambda_destructible(out, lam, op=SK) == 0
    b = np.ones(img.shape, bool)
    b[1:-1, 1:-1] = False
    assert (out[b] == img[b]).all()


@pytest.mark.parametrize("lam", [0, 5, 20])
def test_skeleton_invariants_on_generator_images(lam):
    img = value_noise_image(40, 56, "u8", seed=17)
    out, st = oracle.thin(img, lam, op=SK)
    _skeleton_invariants(img, out, lam)
    assert st["converged"] == 1 and st["lowered"] > 0
    thin_out, _ = oracle.thin(img, lam)
    assert (out >= thin_out).sum() > (out < thin_out).sum()  # end points kept: mostly above the thinning
    if lam == 0:  # only destructible points move at lambda = 0: every section keeps its topology
        levels = sorted(oracle.level_topology(img))
        assert oracle.level_topology(out, levels) == oracle.level_topology(img, levels)


@pytest.mark.parametrize("lam", [0, 10])
def test_paper_minvalue_skeleton_invariants(lam):
    """The paper's own algorithm (minimal value first, Sec. 2.2) reaches a
    fixed point with the same invariants; its image may differ."""
    img = value_noise_image(30, 44, "u8", seed=19)
    out, n = oracle.thin_minvalue(img, lam, op=SK)
    _skeleton_invariants(img, out, lam)
    qout, _ = oracle.thin_queue(img, lam, op=SK)
    _skeleton_invariants(img, qout, lam)


# ---------------------------------------------------------------- (4,8)-adjacency (Sec. 2.1)

A48 = oracle.ADJ_4_8


def test_48_all_masks_against_scipy_labelling():
    for m in range(256):
        g = bf.grid_from_ring(1, [0 if (m >> i) & 1 else 2 for i in range(8)])
        tp_ref, tm_ref, comps = bf.local_numbers(g, adj=1)
        tp, tm, lab = oracle.mask_numbers(m, adj=A48)
        assert (tp, tm) == (tp_ref, tm_ref), m
        got = {}
        for i, l in enumerate(lab):
            if l >= 0:
                got.setdefault(l, set()).add(bf.RING_RC[i])
        assert {frozenset(x) for x in got.values()} == {frozenset(c) for c in comps}, m


def test_48_identity_all_masks():
    """(4,8) in 2-D: T+ = T-- except when no neighbour is lower (T+ = 1,
    T-- = 0) and when every 4-neighbour is lower (T+ = 0, T-- = 1)."""
    four = 0b01010101
    for m in range(256):
        tp, tm, _ = oracle.mask_numbers(m, adj=A48)
        if m == 0:
            assert (tp, tm) == (1, 0)
        elif m & four == four:
            assert (tp, tm) == (0, 1), m
        else:
            assert tp == tm, m


@pytest.mark.parametrize("outer", ["zeros", "ones", "twos", "random"])
def test_48_local_equals_global_all_masks(outer):
    rng = np.random.default_rng(15)
    for m in range(256):
        img = {"zeros": np.zeros((5, 5)), "ones": np.ones((5, 5)), "twos": np.full((5, 5), 2),
               "random": rng.integers(0, 3, (5, 5))}[outer].astype(np.int32)
        img[1:4, 1:4] = bf.grid_from_ring(1, [0 if (m >> i) & 1 else 2 for i in range(8)])
        local, _ = oracle.lowerable(bf.ring_values(img[1:4, 1:4]), 1, 0, adj=A48)
        assert local == oracle.global_destructible(img, 2, 2, adj=A48) == bf.global_destructible(img, 2, 2, adj=1), \
            (m, outer)


def test_48_local_equals_global_random_images():
    rng = np.random.default_rng(41)
    for _ in range(1200):
        img = rng.integers(0, 3, (5, 5)).astype(np.int32)
        for y in range(1, 4):
            for x in range(1, 4):
                local, _ = oracle.lowerable(bf.ring_values(img[y - 1:y + 2, x - 1:x + 2]), img[y, x], 0, adj=A48)
                assert local == oracle.global_destructible(img, x, y, adj=A48), (img, x, y)


def test_48_point_tests_against_reference():
    rng = np.random.default_rng(43)
    for _ in range(3000):
        g = rng.integers(0, 7, (3, 3))
        nb = bf.ring_values(g)
        for lam in (0, 2, 4):
            for rule in (0, 1):
                for op, ref_fn in ((oracle.OP_THIN, bf.point_step), (oracle.OP_SKELETON, bf.skeleton_step)):
                    got = oracle.lowerable(nb, g[1, 1], lam, rule, op=op, adj=A48)
                    ref = ref_fn(g, lam, rule, adj=1)
                    assert got[0] == ref[0], (g, lam, rule, op)
                    if got[0]:
                        assert got[1] == ref[1]


@pytest.mark.parametrize("lam,op", [(0, 0), (2, 0), (0, 1), (3, 1)])
def test_48_schedule_against_python_reference(lam, op):
    rng = np.random.default_rng(300 + lam + 10 * op)
    for _ in range(10):
        h, w = int(rng.integers(3, 9)), int(rng.integers(3, 10))
        img = rng.integers(0, 5, (h, w)).astype(np.int32)
        out, st = oracle.thin(img, lam, op=op, adj=A48)
        assert np.array_equal(out, bf.schedule(img, lam, op=op, adj=1)), img
        assert st["converged"] == 1


@pytest.mark.parametrize("op", [0, 1])
def test_48_lambda0_against_global_brute_force(op):
    rng = np.random.default_rng(23 + op)
    for _ in range(8):
        h, w = int(rng.integers(4, 8)), int(rng.integers(4, 8))
        img = rng.integers(0, 4, (h, w)).astype(np.int32)
        out, _ = oracle.thin(img, 0, op=op, adj=A48)
        assert np.array_equal(out, bf.schedule(img, 0, use_global=True, op=op, adj=1)), img


@pytest.mark.parametrize("lam", [0, 8])
def test_48_invariants_and_topology(lam):
    img = value_noise_image(36, 50, "u8", seed=27)
    out, st = oracle.thin(img, lam, adj=A48)
    assert (out <= img).all() and st["converged"] == 1 and st["lowered"] > 0
    assert oracle.count_lambda_destructible(out, lam, adj=A48) == 0
    if lam == 0:
        levels = sorted(oracle.level_topology(img, adj=A48))
        assert oracle.level_topology(out, levels, adj=A48) == oracle.level_topology(img, levels, adj=A48)
    # the two adjacency pairs are different operators on this image
    assert not np.array_equal(out, oracle.thin(img, lam)[0])


def test_golden_skeleton_and_48_cases():
    """Hand-worked 3x3 cases (tests/golden/skeleton_and_48_cases.json): the
    connectivity numbers under both pairs, whether the centre may be lowered,
    and its final value, for both operators."""
    doc = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "skeleton_and_48_cases.json")))
    adjs = {"8,4": oracle.ADJ_8_4, "4,8": oracle.ADJ_4_8}
    ops = {"thinning": oracle.OP_THIN, "skeleton": oracle.OP_SKELETON}
    assert len(doc["cases"]) >= 4
    for c in doc["cases"]:
        g = np.array(c["grid"])
        nb, ctr = bf.ring_values(g), int(g[1, 1])
        m = sum(1 << i for i, v in enumerate(nb) if v < ctr)
        for a, e in c["expect"].items():
            assert oracle.mask_numbers(m, adj=adjs[a])[:2] == (e["tplus"], e["tminus"]), (c["name"], a)
        for chk in c["checks"]:
            ok, _ = oracle.lowerable(nb, ctr, chk["lam"], op=ops[chk["op"]], adj=adjs[chk["adj"]])
            assert ok == chk["first"], (c["name"], chk)
            out, _ = oracle.thin(g.astype(np.int32), chk["lam"], op=ops[chk["op"]], adj=adjs[chk["adj"]])
            assert out[1, 1] == chk["final"], (c["name"], chk)
