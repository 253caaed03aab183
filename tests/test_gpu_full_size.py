"""GPU parity at full size: the default entry points against the CPU oracle's
stored results on the full-size workloads.

The oracle's results were written by tests/golden/make_full_size_digests.py,
which calls only the oracle and the seeded input generator; each case
records its input recipe, the SHA-256 of the oracle's thinned image, its
number of lowering steps and its last changing phase.  Here every input is
regenerated from its recipe, thinned on the GPU in the launch configuration
the benchmark times (thin_run for single images, one thin_batch call for a
batch, the graph plan for the uneven batch), and compared bit for bit
through the digest and both counts."""
import hashlib
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1603_09180_gb300 import synth, thin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "full_size_digests.json")) as f:
    CASES = json.load(f)["cases"]


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _gen(r):
    return synth.value_noise_image(r["h"], r["w"], r["dtype"], seed=r["seed"], vmax=r["vmax"])


def generate(names):
    """Inputs of the named cases, made in a spawn pool (safe after CUDA is initialised)."""
    recs = [CASES[n] for n in names]
    if len(recs) < 4:
        return [_gen(r) for r in recs]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 2)) as pool:
        return pool.map(_gen, recs, chunksize=4)


def to_dev(a):
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16).copy()).cuda().view(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def expect(name, img_in, got, st):
    r = CASES[name]
    assert digest(img_in) == r["input_sha256"], "%s: input differs from the recorded recipe" % name
    assert st["lowered"] == r["lowered"], name
    assert st["last_change_phase"] == r["last_change_phase"], name
    assert st["converged"] == 1 and st["status"] == 0, name
    assert digest(got) == r["sha256"], "%s: thinned image differs from the oracle's" % name


def test_every_case_is_recorded():
    names = set(CASES)
    assert "single_512_u8_s1603_l0" in names
    assert sum(n.startswith("batch_512_") for n in names) == 192
    assert sum(n.startswith("large_") for n in names) == 4
    assert sum(n.startswith("uneven_") for n in names) == 1024


def test_single_512():
    name = "single_512_u8_s1603_l0"
    img = generate([name])[0]
    t = to_dev(img)
    st = thin.run(t, CASES[name]["lam"])
    expect(name, img, to_host(t), st)


def test_batch192_one_call():
    """All 192 jobs (64 images x lambda {0, 5, 20}) in one thin_batch call, as the benchmark runs them."""
    names = ["batch_512_u8_s%d_l%d" % (s, lam) for s in range(64) for lam in (0, 5, 20)]
    imgs = generate(["batch_512_u8_s%d_l0" % s for s in range(64)])
    work = torch.from_numpy(np.stack([imgs[k // 3] for k in range(192)])).cuda()
    plan = thin.BatchPlan([work[k] for k in range(192)], [CASES[n]["lam"] for n in names])
    sts, rc = plan.run(stats=True)
    assert rc == 0
    out = work.cpu().numpy()
    for k, n in enumerate(names):
        expect(n, imgs[k // 3], out[k], sts[k])


@pytest.mark.parametrize("name,kernel", [("large_4096_u8_s1603_l0", "auto"), ("large_4096_u8_s1603_l30", "auto"),
                                         ("large_4096_u8_s1603_l0", "tiled"), ("large_4096_u8_s1603_l30", "tiled"),
                                         ("large_8192_u16_s1604_l0", "auto"), ("large_8192_u16_s1604_l30", "auto")])
def test_large(name, kernel):
    """4096^2 u8 on the default engine (the wide resident mode) and on the tiled engine; 8192^2 u16
    (0..4095) on the default engine (tiled)."""
    img = generate([name])[0]
    t = to_dev(img)
    st = thin.run(t, CASES[name]["lam"], kernel=kernel)
    expect(name, img, to_host(t), st)
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("runner", ["batch", "graph"])
def test_uneven_1024(runner):
    """The 1024 uneven u8 images (sides 64..2048, lambda {0, 10, 25}) in one call: a thin_batch call,
    and the graph-captured plan with the autotuned tiled group."""
    names = ["uneven_%04d" % i for i in range(1024)]
    imgs = generate(names)
    work = [to_dev(a) for a in imgs]
    lams = [CASES[n]["lam"] for n in names]
    plan = thin.BatchPlan(work, lams) if runner == "batch" else thin.GraphPlan(work, lams)
    sts, rc = plan.run(stats=True)
    assert rc == 0
    for n, a, t, st in zip(names, imgs, work, sts):
        expect(n, a, to_host(t), st)
    if runner == "graph":
        plan.close()
