"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Integer work, so the bar is bit-exact images, plus equal lowering counts and
equal last changing phase.  Inputs come from the seeded generator."""
import numpy as np
import pytest

import oracle
from paper_1603_09180_gb300 import synth, thin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def to_dev(a):
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16).copy()).cuda().view(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def check(img, lam, rule="max", **kw):
    t = to_dev(img)
    st = thin.run(t, lam, rule=rule, **kw)
    torch.cuda.synchronize()
    ref, rst = oracle.thin(img, lam, oracle.RULE_MAX if rule == "max" else oracle.RULE_MIN,
                           start_phase=kw.get("start_phase", 0), max_phases=kw.get("max_phases", -1),
                           op=oracle.OP_SKELETON if kw.get("op") == "skeleton" else oracle.OP_THIN,
                           adj=kw.get("adj", thin.ADJ_8_4))
    got = to_host(t)
    assert np.array_equal(got, ref), "mismatch at %s" % (np.argwhere(got != ref)[:5].tolist(),)
    assert st["lowered"] == rst["lowered"]
    assert st["last_change_phase"] == rst["last_change_phase"]
    if kw.get("max_phases", -1) < 0:
        assert st["converged"] == 1 and st["rc"] == 0
    return st, rst


SHAPES = [(3, 3), (3, 40), (40, 3), (5, 7), (17, 33), (64, 64), (65, 129), (100, 231), (128, 200)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("lam", [0, 6])
def test_naive_matches_oracle(shape, lam):
    img = synth.value_noise_image(*shape, "u8", seed=shape[0] * 7 + shape[1])
    check(img, lam, kernel="naive")


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("lam", [0, 5, 20])
def test_engines_match_oracle(shape, lam, kernel):
    img = synth.value_noise_image(*shape, "u8", seed=shape[0] * 3 + shape[1])
    check(img, lam, kernel=kernel)


@pytest.mark.parametrize("tile,halo", [((16, 8), 3), ((16, 16), 4), ((32, 16), 8), ((48, 40), 5), ((64, 64), 8),
                                       ((128, 64), 6), ((224, 32), 7), ((32, 128), 3)])
@pytest.mark.parametrize("dt", ["u8", "u16"])
def test_tiled_tile_shapes(tile, halo, dt):
    img = synth.value_noise_image(150, 170, dt, seed=halo * 11 + tile[0])
    lam = 7 if dt == "u8" else 100
    check(img, lam, tile=tile, halo=halo, kernel="tiled")


@pytest.mark.parametrize("rule", ["max", "min"])
@pytest.mark.parametrize("kernel", ["naive", "tiled", "resident"])
def test_rules(rule, kernel):
    img = synth.value_noise_image(90, 110, "u8", seed=31)
    check(img, 12, rule=rule, kernel=kernel)


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
@pytest.mark.parametrize("dt,vmax,lam", [("u16", 4095, 0), ("u16", 4095, 30), ("u16", 65535, 700), ("u8", 255, 255)])
def test_value_ranges(dt, vmax, lam, kernel):
    img = synth.value_noise_image(96, 120, dt, seed=vmax + lam, vmax=vmax)
    check(img, lam, kernel=kernel)


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
def test_white_noise_worst_case(kernel):
    img = synth.uniform_noise_image(130, 150, "u8", seed=4)
    check(img, 0, kernel=kernel)
    check(img, 40, kernel=kernel)


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
def test_unaligned_pitch_and_offset(kernel):
    """Rows that are not 16-byte aligned: internal buffers (tiled) or plain loads (resident)."""
    img = synth.value_noise_image(70, 90, "u8", seed=2)
    big = np.zeros((80, 101), np.uint8)
    big[3:73, 5:95] = img
    t = to_dev(big)
    view = t[3:73, 5:95]
    st = thin.run(view, 9, kernel=kernel)
    torch.cuda.synchronize()
    ref, _ = oracle.thin(img, 9)
    out = to_host(t)
    assert np.array_equal(out[3:73, 5:95], ref)
    mask = np.ones_like(big, bool)
    mask[3:73, 5:95] = False
    assert np.array_equal(out[mask], big[mask])  # nothing outside the view is touched
    assert st["converged"] == 1


@pytest.mark.parametrize("kernel", ["naive", "tiled", "resident"])
@pytest.mark.parametrize("cap", [1, 4, 7, 13, 40])
def test_cap_and_resume(kernel, cap):
    img = synth.value_noise_image(80, 96, "u8", seed=12)
    full, _ = oracle.thin(img, 10)
    t = to_dev(img)
    st = thin.run(t, 10, kernel=kernel, max_phases=cap)
    torch.cuda.synchronize()
    part_ref, pst = oracle.thin(img, 10, max_phases=cap)
    assert np.array_equal(to_host(t), part_ref)
    if not st["converged"]:
        assert st["end_phase"] == cap and st["rc"] == thin.THIN_ERR_NOT_CONVERGED
    st2 = thin.run(t, 10, kernel=kernel, start_phase=cap)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t), full)
    assert st["lowered"] + st2["lowered"] == oracle.thin(img, 10)[1]["lowered"]


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
def test_start_phase_offsets(kernel):
    img = synth.value_noise_image(60, 75, "u8", seed=8)
    for g in (1, 2, 3, 6):
        check(img, 4, start_phase=g, kernel=kernel)


@pytest.mark.parametrize("kernel", ["auto", "tiled"])
def test_batch_mixed_equals_alone(kernel):
    rng = np.random.default_rng(0)
    imgs, lams, refs = [], [], []
    for k in range(14):
        h, w = int(rng.integers(3, 260)), int(rng.integers(3, 300))
        dt = "u16" if k % 3 == 0 else "u8"
        img = synth.value_noise_image(h, w, dt, seed=100 + k)
        lam = int(rng.choice([0, 10, 25])) * (16 if dt == "u16" else 1)
        imgs.append(img)
        lams.append(lam)
        refs.append(oracle.thin(img, lam))
    if kernel == "auto":  # one image too large for a cluster's shared memory: both engines in one call
        big = synth.value_noise_image(1000, 2100, "u8", seed=99)
        imgs.append(big)
        lams.append(0)
        refs.append(oracle.thin(big, 0))
    ts = [to_dev(a) for a in imgs]
    sts, rc = thin.batch(ts, lams, kernel=kernel)
    torch.cuda.synchronize()
    assert rc == 0
    for t, (ref, rst), st in zip(ts, refs, sts):
        assert np.array_equal(to_host(t), ref)
        assert st["lowered"] == rst["lowered"] and st["last_change_phase"] == rst["last_change_phase"]


def test_deterministic_repeats():
    img = synth.value_noise_image(200, 260, "u8", seed=77)
    outs = []
    for _ in range(3):
        t = to_dev(img)
        thin.run(t, 15)
        torch.cuda.synchronize()
        outs.append(to_host(t))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
def test_config1_full_size(kernel):
    """512 x 512 u8, lambda = 0, seed 1603: bit-exact at full size."""
    img = synth.value_noise_image(512, 512, "u8", seed=1603)
    check(img, 0, kernel=kernel)


@pytest.mark.parametrize("shape,dt,lam", [((200, 300), "u8", 9), ((512, 512), "u8", 5), ((700, 700), "u8", 0),
                                          ((1024, 1024), "u8", 0), ((512, 512), "u16", 0), ((333, 250), "u16", 7),
                                          ((12, 20000), "u8", 5)])  # 8 blocks of 2 own rows: halo of 2
def test_resident_cluster_sizes(shape, dt, lam):
    """Images that need 1, 2, 4 and 8 blocks per cluster, alone and in a batch (a single
    image is spread over a wider cluster, down to 32 rows per block)."""
    img = synth.value_noise_image(*shape, dt, seed=shape[0] + shape[1])
    check(img, lam, kernel="resident")
    ref, rst = oracle.thin(img, lam)
    ts = [to_dev(img) for _ in range(3)]
    sts, rc = thin.batch(ts, [lam] * 3, kernel="resident")
    torch.cuda.synchronize()
    for t, st in zip(ts, sts):
        assert np.array_equal(to_host(t), ref) and st["lowered"] == rst["lowered"]


def test_timeout_reports_status_and_context_survives(monkeypatch):
    """A grid barrier that can never complete (one block does not arrive)
    gives up after its time limit and reports THIN_ERR_TIMEOUT; the next call
    on the same context works."""
    monkeypatch.setenv("THIN_TIMEOUT_NS", "50000000")
    img = synth.value_noise_image(200, 200, "u8", seed=1)
    t = to_dev(img)
    st = thin.run(t, 0, debug=1, check=False, kernel="tiled")
    torch.cuda.synchronize()
    assert st["rc"] == thin.THIN_ERR_TIMEOUT and st["status"] == thin.THIN_ERR_TIMEOUT
    monkeypatch.delenv("THIN_TIMEOUT_NS")
    check(img, 0, kernel="tiled")


def test_tested_counts():
    """The naive engine tests every interior point of the phase's parity; the
    others test a subset, never more."""
    img = synth.value_noise_image(130, 170, "u8", seed=41)
    st_n, rst = check(img, 6, kernel="naive")
    assert st_n["tested"] == st_n["phases"] * 128 * 168 // 4
    for kernel in ("tiled", "resident"):
        st, _ = check(img, 6, kernel=kernel)
        assert 0 < st["tested"] <= st_n["tested"] + 4 * 128 * 168  # the last quiet phases may run past


# ---------------------------------------------------------------- lambda-skeleton (Sec. 2.2)

@pytest.mark.parametrize("kernel", ["naive", "tiled", "resident"])
@pytest.mark.parametrize("shape", [(3, 40), (17, 33), (65, 129), (128, 200)])
@pytest.mark.parametrize("lam", [0, 5, 20])
def test_skeleton_matches_oracle(shape, lam, kernel):
    img = synth.value_noise_image(*shape, "u8", seed=shape[0] * 5 + shape[1] + lam)
    check(img, lam, kernel=kernel, op="skeleton")


@pytest.mark.parametrize("kernel", ["naive", "tiled", "resident"])
@pytest.mark.parametrize("dt,vmax,lam,rule", [("u16", 4095, 0, "max"), ("u16", 4095, 30, "min"), ("u8", 255, 255, "max"),
                                              ("u8", 255, 12, "min")])
def test_skeleton_value_ranges_and_rules(dt, vmax, lam, rule, kernel):
    img = synth.value_noise_image(96, 120, dt, seed=vmax + lam + 3, vmax=vmax)
    check(img, lam, rule=rule, kernel=kernel, op="skeleton")


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
def test_skeleton_lines_and_peaks(kernel):
    """Thin bright lines and isolated peaks of known contrast (white noise below
    them): lines with contrast above lambda keep their end points."""
    rng = np.random.default_rng(6)
    img = rng.integers(0, 30, (120, 160)).astype(np.uint8)
    for k in range(10):
        y, x = int(rng.integers(5, 110)), int(rng.integers(5, 120))
        img[y, x:x + 30] = 60 + 15 * k
        img[int(rng.integers(2, 118)), int(rng.integers(2, 158))] = 40 + 20 * k
    for lam in (0, 50, 120):
        check(img, lam, kernel=kernel, op="skeleton")
        check(img, lam, kernel=kernel, op="skeleton", max_phases=6)


def test_skeleton_batch_and_plan_match_oracle():
    imgs = [synth.value_noise_image(h, w, dt, seed=h + w) for h, w, dt in
            [(40, 50, "u8"), (300, 200, "u8"), (90, 70, "u16"), (700, 650, "u8"), (1000, 2100, "u8")]]
    lams = [0, 10, 64, 5, 3]
    refs = [oracle.thin(a, l, op=oracle.OP_SKELETON) for a, l in zip(imgs, lams)]
    ts = [to_dev(a) for a in imgs]
    sts, rc = thin.batch(ts, lams, op="skeleton")
    assert rc == 0
    for t, (ref, rst), st in zip(ts, refs, sts):
        assert np.array_equal(to_host(t), ref) and st["lowered"] == rst["lowered"]
    ts = [to_dev(a) for a in imgs]
    plan = thin.GraphPlan(ts, lams, op="skeleton")
    sts, rc = plan.run(stats=True)
    assert rc == 0
    for t, (ref, rst), st in zip(ts, refs, sts):
        assert np.array_equal(to_host(t), ref) and st["lowered"] == rst["lowered"]
    plan.close()


# ---------------------------------------------------------------- (4,8)-adjacency (Sec. 2.1)

@pytest.mark.parametrize("kernel", ["naive", "tiled", "resident"])
@pytest.mark.parametrize("dt", ["u8", "u16"])
@pytest.mark.parametrize("op", ["thinning", "skeleton"])
@pytest.mark.parametrize("lam", [0, 9])
def test_48_matches_oracle(kernel, dt, op, lam):
    img = synth.value_noise_image(70, 133, dt, seed=48 + lam)
    check(img, lam * (16 if dt == "u16" else 1), kernel=kernel, op=op, adj=thin.ADJ_4_8)


@pytest.mark.parametrize("kernel", ["tiled", "resident"])
def test_48_sizes_noise_and_cap(kernel):
    for shape in [(3, 3), (5, 40), (64, 64), (129, 65)]:
        check(synth.value_noise_image(*shape, "u8", seed=sum(shape)), 4, kernel=kernel, adj=thin.ADJ_4_8)
    noise = synth.uniform_noise_image(90, 110, "u8", seed=3)
    check(noise, 0, kernel=kernel, adj=thin.ADJ_4_8)
    check(noise, 30, kernel=kernel, adj=thin.ADJ_4_8, max_phases=7)


def test_48_batch_plan_and_full_size():
    imgs = [synth.value_noise_image(h, w, dt, seed=h * w) for h, w, dt in
            [(50, 60, "u8"), (512, 512, "u8"), (300, 260, "u16"), (1000, 2100, "u8")]]
    lams = [3, 0, 40, 5]
    refs = [oracle.thin(a, l, adj=oracle.ADJ_4_8) for a, l in zip(imgs, lams)]
    for mk in ("batch", "plan"):
        ts = [to_dev(a) for a in imgs]
        if mk == "batch":
            sts, rc = thin.batch(ts, lams, adj=thin.ADJ_4_8)
        else:
            plan = thin.GraphPlan(ts, lams, adj=thin.ADJ_4_8)
            sts, rc = plan.run(stats=True)
            plan.close()
        assert rc == 0
        for t, (ref, rst), st in zip(ts, refs, sts):
            assert np.array_equal(to_host(t), ref), mk
            assert st["lowered"] == rst["lowered"]


# ---------------------------------------------------------------- wide resident mode

@pytest.mark.parametrize("shape,dt,lam", [((1400, 1400), "u8", 0), ((1400, 1400), "u8", 3), ((1000, 1100), "u16", 0),
                                          ((200, 12000), "u8", 2), ((1300, 1500), "u8", 0), ((2100, 1900), "u8", 0),
                                          ((1500, 1400), "u16", 0)])
def test_wide_matches_oracle(shape, dt, lam):
    """Images larger than an 8-block cluster's shared memory: held by one
    cluster of 16 where the device runs such clusters and the image fits one,
    else by several clusters of one launch (the wide mode: boundary rows cross
    through global memory every 8 phases).  The default engine and the
    resident engine forced both keep the image on chip."""
    img = synth.value_noise_image(*shape, dt, seed=shape[0] + 3 * shape[1] + lam)
    ref, rst = oracle.thin(img, lam)
    for kernel in ("auto", "resident"):
        t = to_dev(img)
        st = thin.run(t, lam, kernel=kernel)
        torch.cuda.synchronize()
        assert st["tiles_visited"] == 0  # the resident engine ran, not the tiled one
        assert np.array_equal(to_host(t), ref), kernel
        assert st["lowered"] == rst["lowered"] and st["last_change_phase"] == rst["last_change_phase"]


@pytest.mark.parametrize("cap", [3, 13])
def test_wide_cap_and_resume(cap):
    img = synth.value_noise_image(1400, 1400, "u8", seed=77)
    check(img, 4, kernel="resident", max_phases=cap)
    full, _ = oracle.thin(img, 4)
    t = to_dev(img)
    thin.run(t, 4, kernel="resident", max_phases=cap)
    thin.run(t, 4, kernel="resident", start_phase=cap)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t), full)


@pytest.mark.parametrize("dt,lam", [("u8", 30), ("u16", 0)])
def test_wide_full_size_equals_tiled(dt, lam):
    """4096 x 4096 u8 and 2800 x 2800 u16: the wide mode and the tiled engine give
    the same image (both bit-exact to the oracle on smaller cases); the result
    is a fixed point of the oracle's test and lies below the input."""
    shape = (4096, 4096) if dt == "u8" else (2800, 2800)
    img = synth.value_noise_image(*shape, dt, seed=1603)
    a, b = to_dev(img), to_dev(img)
    sa = thin.run(a, lam, kernel="resident")
    sb = thin.run(b, lam, kernel="tiled")
    torch.cuda.synchronize()
    assert sa["tiles_visited"] == 0 and sb["tiles_visited"] > 0
    assert torch.equal(a, b)
    assert sa["lowered"] == sb["lowered"] and sa["last_change_phase"] == sb["last_change_phase"]
    out = to_host(a)
    assert (out <= img).all()
    assert oracle.count_lambda_destructible(out, lam) == 0
