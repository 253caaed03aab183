"""Batch plans (thin_plan_*): a batch prepared once and replayed as one CUDA
graph.  Results must be bit-exact to the CPU oracle on every replay, with the
resident engine's cluster-size groups running side by side and the tiled
engine after them."""
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


def mixed(seed):
    rng = np.random.default_rng(seed)
    imgs, lams = [], []
    for k in range(10):
        h, w = int(rng.integers(3, 300)), int(rng.integers(3, 300))
        dt = "u16" if k % 3 == 0 else "u8"
        imgs.append(synth.value_noise_image(h, w, dt, seed=seed * 100 + k))
        lams.append(int(rng.choice([0, 10, 25])) * (16 if dt == "u16" else 1))
    # one image per wider cluster, one for the tiled engine, one with no interior
    imgs += [synth.value_noise_image(700, 700, "u8", seed=seed + 1), synth.value_noise_image(512, 512, "u16", seed=seed + 2),
             synth.value_noise_image(1000, 2100, "u8", seed=seed + 3), synth.value_noise_image(2, 40, "u8", seed=4)]
    lams += [5, 0, 0, 3]
    return imgs, lams


def test_plan_replays_match_oracle():
    imgs, lams = mixed(1)
    refs = [oracle.thin(a, l) for a, l in zip(imgs, lams)]
    pristine = [to_dev(a) for a in imgs]
    work = [p.clone() for p in pristine]
    plan = thin.GraphPlan(work, lams)
    for rep in range(3):
        for w, p in zip(work, pristine):
            w.copy_(p)
        sts, rc = plan.run(stats=True)
        assert rc == 0
        for t, (ref, rst), st in zip(work, refs, sts):
            assert np.array_equal(to_host(t), ref), rep
            assert st["lowered"] == rst["lowered"] and st["last_change_phase"] == rst["last_change_phase"]
            assert st["converged"] == 1
    # a replay on the thinned images changes nothing: they are at the fixed point
    sts, rc = plan.run(stats=True)
    assert rc == 0 and all(s["lowered"] == 0 for s in sts)
    for t, (ref, _) in zip(work, refs):
        assert np.array_equal(to_host(t), ref)
    plan.close()


def test_plan_equals_batch_call_and_cap():
    imgs, lams = mixed(2)
    a = [to_dev(x) for x in imgs]
    b = [to_dev(x) for x in imgs]
    sts_b, rc_b = thin.batch(b, lams, max_phases=9, start_phase=2)
    plan = thin.GraphPlan(a, lams, max_phases=9, start_phase=2)
    sts_a, rc_a = plan.run(stats=True)
    torch.cuda.synchronize()
    assert rc_a == rc_b
    for x, y, sa, sb in zip(a, b, sts_a, sts_b):
        assert torch.equal(x, y)
        assert sa == sb
    for img, lam, x in zip(imgs, lams, a):
        ref, _ = oracle.thin(img, lam, start_phase=2, max_phases=9)
        assert np.array_equal(to_host(x), ref)
    plan.close()


def test_plan_of_images_without_interior():
    t = [to_dev(np.zeros((2, 9), np.uint8)), to_dev(np.zeros((0, 5), np.uint8))]
    plan = thin.GraphPlan(t, [0, 0])
    sts, rc = plan.run(stats=True)
    assert rc == 0 and all(s["converged"] == 1 and s["phases"] == 0 for s in sts)
    plan.close()


@pytest.mark.parametrize("dt,lam", [("u8", 12), ("u16", 100)])
def test_autotune_picks_a_valid_shape_and_leaves_the_image(dt, lam):
    img = synth.value_noise_image(300, 420, dt, seed=9)
    t = to_dev(img)
    cfg, ms = thin.autotune(t, lam, trial_phases=64)
    assert ms > 0 and cfg["tile"][0] % 16 == 0 and cfg["halo"] >= 3
    assert np.array_equal(to_host(t), img)  # trials ran on a copy
    st = thin.run(t, lam, kernel="tiled", **cfg)
    torch.cuda.synchronize()
    ref, rst = oracle.thin(img, lam)
    assert np.array_equal(to_host(t), ref) and st["lowered"] == rst["lowered"]


def test_plan_autotunes_its_tiled_images():
    """A plan whose images go to the tiled engine picks their tile shape and halo
    by timing (on a scratch copy); the replays stay bit-exact to the oracle."""
    imgs = [synth.value_noise_image(h, w, "u8", seed=h + w) for h, w in [(300, 420), (257, 190), (64, 700)]]
    lams = [6, 0, 12]
    refs = [oracle.thin(a, l) for a, l in zip(imgs, lams)]
    pristine = [to_dev(a) for a in imgs]
    work = [p.clone() for p in pristine]
    plan = thin.GraphPlan(work, lams, kernel="tiled")
    tw, th, halo = plan.tiling()
    assert tw % 16 == 0 and tw >= 16 and th >= 8 and 3 <= halo <= 8
    for t, p in zip(work, pristine):
        assert torch.equal(t, p)  # the trials did not touch the images
    for _ in range(2):
        for t, p in zip(work, pristine):
            t.copy_(p)
        sts, rc = plan.run(stats=True)
        assert rc == 0
        for t, (ref, rst), st in zip(work, refs, sts):
            assert np.array_equal(to_host(t), ref) and st["lowered"] == rst["lowered"]
    fixed = thin.GraphPlan(work, lams, kernel="tiled", tile=(32, 32), halo=5)
    assert fixed.tiling() == (0, 0, 0)  # the caller's shape is used as given
    plan.close()
    fixed.close()
