"""Serving (thin_serve_*): continuous batching under a device-memory budget.

Requests of mixed sizes, dtypes and lambdas go through one server from
several host threads; every result must be bit-exact to what thin_run gives
the same image alone (integer work) and to the CPU oracle.  Each image is
retired as soon as it is finished, so a slow image does not hold back small
ones admitted with it.  Admission limits (queue cap, budget) are checked
too.  Lambda applies to pixel values as given, for u8 and u16 alike."""
import multiprocessing as mp
import os
import threading

import numpy as np
import pytest

import oracle
from paper_1603_09180_gb300 import synth, thin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def alone(img, lam):
    if img.dtype == np.uint16:
        t = torch.from_numpy(img.view(np.int16).copy()).cuda().view(torch.uint16)
    else:
        t = torch.from_numpy(img.copy()).cuda()
    st = thin.run(t, lam)
    torch.cuda.synchronize()
    out = t.view(torch.int16).cpu().numpy().view(np.uint16) if img.dtype == np.uint16 else t.cpu().numpy()
    return out, st


def mixed_requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        dt = "u16" if k % 2 else "u8"
        h, w = (int(np.exp(rng.uniform(np.log(8), np.log(600)))) for _ in range(2))
        lam = int(rng.choice([0, 10]))
        reqs.append((synth.value_noise_image(h, w, dt, seed=seed * 1000 + k), lam))
    # two images too large for one cluster's shared memory (the tiled engine), and two with no interior
    reqs.append((synth.value_noise_image(1500, 1300, "u8", seed=seed + 7), 10))
    reqs.append((synth.value_noise_image(1000, 1000, "u16", seed=seed + 8), 0))
    reqs.append((synth.value_noise_image(2, 50, "u8", seed=1), 5))
    reqs.append((np.zeros((0, 0), np.uint8), 0))
    return reqs


def _oracle(args):
    img, lam = args
    return oracle.thin(img, lam)


def oracle_all(pairs):
    """The oracle on every (image, lambda), in a spawn pool (safe after CUDA is initialised)."""
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 2)) as pool:
        return pool.map(_oracle, pairs, chunksize=1)


def collect(srv, n):
    got = {}
    while len(got) < n:
        t = srv.wait_any(20000)
        assert t is not None, "no request finished within 20 s"
        done, out, st, rc = srv.poll(t)
        assert done and rc == thin.THIN_OK, rc
        got[t] = (out, st)
    return got


@pytest.mark.parametrize("slots", [12, 2])
def test_serve_mix_from_three_threads_equals_alone(slots):
    """With 2 slots, batches are small and the lanes run different image sizes at once."""
    reqs = mixed_requests(45, 5 + slots)
    tickets = [None] * len(reqs)
    with thin.Server(1 << 30, max_slots=slots, queue_cap=len(reqs)) as srv:
        def client(idx):
            for i in idx:
                tickets[i] = srv.submit(*reqs[i])
        th = [threading.Thread(target=client, args=(range(k, len(reqs), 3),)) for k in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = collect(srv, len(reqs))
    assert sorted(got) == sorted(tickets)
    # the oracle on every image up to 600 x 600 (the two larger ones are checked against thin_run here
    # and against the oracle at full size elsewhere)
    real = [k for k, (img, _) in enumerate(reqs) if img.shape[0] >= 3 and img.shape[1] >= 3]
    small = [k for k in real if reqs[k][0].size <= 600 * 600]
    orc = dict(zip(small, oracle_all([reqs[k] for k in small])))
    for k, ((img, lam), t) in enumerate(zip(reqs, tickets)):
        out, st = got[t]
        if k not in real:
            assert np.array_equal(out, img) and st["converged"] == 1
            continue
        ref, st1 = alone(img, lam)
        assert np.array_equal(out, ref), (img.shape, img.dtype, lam)
        assert st["lowered"] == st1["lowered"] and st["last_change_phase"] == st1["last_change_phase"]
        assert st["converged"] == 1
        if k in orc:
            oref, ost = orc[k]
            assert np.array_equal(out, oref) and st["lowered"] == ost["lowered"]
            assert st["last_change_phase"] == ost["last_change_phase"]


def test_serve_small_images_do_not_wait_for_a_slow_one():
    """One slow image (512^2, lambda 20, about 4000 phases) and 40 small ones submitted right after it:
    every small one finishes before the slow one, whether a lane admitted them with it or not."""
    slow = synth.value_noise_image(512, 512, "u8", seed=38)
    small = [synth.value_noise_image(48, 64, "u8", seed=100 + k) for k in range(40)]
    with thin.Server(1 << 30, max_slots=8 * 64, queue_cap=64) as srv:
        ts = srv.submit(slow, 20)
        tk = [srv.submit(im, 0) for im in small]
        order, outs = [], {}
        while len(order) < 1 + len(small):
            t = srv.wait_any(20000)
            assert t is not None
            done, out, st, rc = srv.poll(t)
            assert done and rc == 0
            order.append(t)
            outs[t] = out
    # the results are checked after the server is gone: a synchronising call from this thread while
    # the slow image runs could hold up the lanes' launches and change the order being tested
    assert order[-1] == ts
    for t, out in outs.items():
        img, lam = (slow, 20) if t == ts else (small[tk.index(t)], 0)
        ref, _ = alone(img, lam)
        assert np.array_equal(out, ref)


def test_serve_queue_cap_and_budget():
    big = synth.value_noise_image(900, 1000, "u8", seed=3)
    with thin.Server(64 << 20, max_slots=1, queue_cap=1) as srv:
        tickets, again = [], 0
        for _ in range(12):
            try:
                tickets.append(srv.submit(big, 25))
            except thin.ThinError as e:
                assert e.code == thin.THIN_EAGAIN
                again += 1
        assert again >= 1 and len(tickets) >= 1  # one running, one waiting at most while the rest arrive
        got = collect(srv, len(tickets))
        ref, _ = alone(big, 25)
        for t in tickets:
            assert np.array_equal(got[t][0], ref)
    with thin.Server(1 << 20, max_slots=4, queue_cap=4) as srv:
        with pytest.raises(thin.ThinError) as ei:
            srv.submit(big, 0)  # charged more than the whole budget
        assert ei.value.code == thin.THIN_ERR_TOO_LARGE


def test_serve_budget_admits_one_at_a_time():
    """A budget that holds one image at a time still finishes everything, in order."""
    imgs = [synth.value_noise_image(300, 340, "u8", seed=s) for s in range(6)]
    one = 2 * 352 * 300 + 340 * 300 // 4 + (64 << 10)  # the charge of one 300 x 340 u8 image (rows padded to 352 B)
    with thin.Server(one + 1000, max_slots=8, queue_cap=8) as srv:
        tickets = [srv.submit(im, 5) for im in imgs]
        order = []
        while len(order) < len(imgs):
            t = srv.wait_any(20000)
            assert t is not None
            done, out, st, rc = srv.poll(t)
            assert done and rc == 0
            order.append(t)
            ref, _ = alone(imgs[tickets.index(t)], 5)
            assert np.array_equal(out, ref)
    assert order == tickets  # one admitted at a time, first come first served
