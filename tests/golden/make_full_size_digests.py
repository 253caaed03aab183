"""Writes full_size_digests.json: the CPU oracle's results on the full-size
workloads, as SHA-256 digests of the thinned images plus the oracle's counts.

Calls only ``oracle`` (the plain CPU restatement of Sec. 2.1-2.2) and the
seeded input generator ``synth``; nothing here touches the CUDA library.
The GPU parity tests regenerate each input from its recorded recipe, thin it
with the default entry points and compare the digest, ``lowered`` and
``last_change_phase`` with the values stored here.

Cases (default options: lambda-thinning, F^-(c) = max over c, (8,4)):
  single  512x512 u8, seed 1603, lambda 0
  batch   64 images 512x512 u8 (seeds 0..63) x lambda {0, 5, 20}
  large   4096x4096 u8 (seed 1603) and 8192x8192 u16 in 0..4095 (seed 1604),
          lambda {0, 30}
  uneven  the 1024 jobs of synth.uneven_batch_specs() (u8, sides 64..2048,
          lambda {0, 10, 25})

The file is rewritten after every finished case, so an interrupted run
resumes where it stopped.  Usage:
  python tests/golden/make_full_size_digests.py [--jobs N] [--only PREFIX ...]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "full_size_digests.json")


def cases():
    """Every case as (name, recipe).  A recipe names the generator call and lambda."""
    sys.path.insert(0, ROOT)
    from paper_1603_09180_gb300 import synth
    out = [("single_512_u8_s1603_l0", dict(h=512, w=512, dtype="u8", seed=1603, vmax=255, lam=0))]
    for seed in range(64):
        for lam in (0, 5, 20):
            out.append(("batch_512_u8_s%d_l%d" % (seed, lam), dict(h=512, w=512, dtype="u8", seed=seed, vmax=255,
                                                                 lam=lam)))
    for lam in (0, 30):
        out.append(("large_4096_u8_s1603_l%d" % lam, dict(h=4096, w=4096, dtype="u8", seed=1603, vmax=255, lam=lam)))
        out.append(("large_8192_u16_s1604_l%d" % lam, dict(h=8192, w=8192, dtype="u16", seed=1604, vmax=4095,
                                                            lam=lam)))
    for i, (h, w, lam, seed) in enumerate(synth.uneven_batch_specs()):
        out.append(("uneven_%04d" % i, dict(h=h, w=w, dtype="u8", seed=seed, vmax=255, lam=lam, index=i)))
    return out


def digest(img) -> str:
    """SHA-256 of the image's bytes, row-major, in its own dtype (little-endian)."""
    import numpy as np
    a = np.ascontiguousarray(img)
    if a.dtype.byteorder == ">":
        a = a.byteswap().view(a.dtype.newbyteorder("<"))
    return hashlib.sha256(a.tobytes()).hexdigest()


def run_case(item):
    name, r = item
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1603_09180_gb300 import synth
    img = synth.value_noise_image(r["h"], r["w"], r["dtype"], seed=r["seed"], vmax=r["vmax"])
    t0 = time.time()
    res, st = oracle.thin(img, r["lam"])
    dt = time.time() - t0
    rec = dict(r)
    rec.update(sha256=digest(res), input_sha256=digest(img), lowered=st["lowered"],
               last_change_phase=st["last_change_phase"], phases=st["phases"], rounds=st["rounds"],
               oracle_s=round(dt, 1))
    return name, rec


def cost(recipe) -> float:
    """A rough ordering key: longest first, so the big cases start at once."""
    return recipe["h"] * recipe["w"] * (1.0 + recipe["lam"]) * (2.0 if recipe["dtype"] == "u16" else 1.0)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--only", nargs="*", default=None, help="case-name prefixes to compute")
    args = ap.parse_args(argv)
    done = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            done = json.load(f)["cases"]
    todo = [(n, r) for n, r in cases() if n not in done and (not args.only or any(n.startswith(p) for p in args.only))]
    todo.sort(key=lambda c: -cost(c[1]))
    print("%d cases to compute, %d already stored" % (len(todo), len(done)), flush=True)
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        for name, rec in pool.imap_unordered(run_case, todo):
            done[name] = rec
            body = {"about": "CPU oracle (oracle.thin, default options) on seeded synth inputs; written by "
                             "tests/golden/make_full_size_digests.py. sha256 is over the thinned image's bytes, "
                             "row-major, little-endian, in the input dtype.",
                    "cases": dict(sorted(done.items()))}
            tmp = OUT + ".tmp"
            with open(tmp, "w") as f:
                json.dump(body, f, indent=0, sort_keys=True)
            os.replace(tmp, OUT)
            print("%s  %.1f s  rounds %d" % (name, rec["oracle_s"], rec["rounds"]), flush=True)


if __name__ == "__main__":
    main()
