"""FP64 oracle iterates of the precision workload, on a seeded sample of voxels.

TEST INFRASTRUCTURE ONLY: it runs the oracle (and the seeded input generators); the
product path never reads what it writes.

The precision workload is the grid (256, 1024, 256) with a 512 x 512 detector at 0.4 mm,
the medium phantom family and 30 SART sweeps (Eq. 7, one view per subset, lambda 0.5,
warm start, ROI weights).  At 360 views the oracle would need hours per sweep, so this
script runs a crop of the views (every 90th: 4 views, full grid and detector) and keeps,
at sweeps 1, 10 and 30, the oracle's iterate on 2^18 voxels drawn without replacement
from a seeded generator.  The relative L2 of a GPU iterate against the oracle is then
estimated on that sample.

The oracle runs once per stored input precision: the FP32 sinogram and warm start, and
their FP16 and BF16 roundings (round to nearest even), each widened to FP64 exactly, so
that the GPU's 16-bit path is compared with the exact SART of the very inputs it holds.

Output: ``oracle/_cache/precision_<hash>.npz``; the hash covers every setting below.
Usage: ``python -m oracle.precision_reference [--threads N]``.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

VIEW_STEP = 90                  # views 0, 90, 180, 270 of the 360
SWEEPS = (1, 10, 30)
N_SAMPLE = 1 << 18
SAMPLE_SEED = 20051197 + 77
POISSON_SEED = 300
I0 = 1.0e4
LAMBDA = 0.5
DTYPES = ("f32", "f16", "bf16")


def crop_scan():
    from paper_2005_11976_gb300 import synth
    full = synth.precision_scan(synth.rng_for("precision"))
    return dataclasses.replace(full, angles=full.angles[::VIEW_STEP])


def settings() -> dict:
    s = crop_scan()
    f = s.fields()
    f["angles"] = [float(a) for a in f["angles"]]
    return {"scan": f, "view_step": VIEW_STEP, "sweeps": list(SWEEPS), "n_sample": N_SAMPLE,
            "sample_seed": SAMPLE_SEED, "poisson_seed": POISSON_SEED, "i0": I0, "lambda": LAMBDA,
            "dtypes": list(DTYPES), "phantom": "synth.part_phantom, removed insert from rng_for('precision')"}


def cache_path() -> str:
    key = json.dumps(settings(), sort_keys=True, default=str).encode()
    with open(os.path.join(HERE, "cyl_oracle.c"), "rb") as f:     # the oracle's arithmetic too
        key += f.read()
    h = hashlib.sha256(key).hexdigest()[:16]
    return os.path.join(HERE, "_cache", f"precision_{h}.npz")


def inputs():
    """(scan, FP64 line integrals of the crop, warm start, ROI weights, sample indices): the
    data are the oracle's own projection of the part with one insert removed, Poisson
    counts at I0 (seeded) and their log transform."""
    import oracle
    from paper_2005_11976_gb300 import synth
    s = crop_scan()
    rng = synth.rng_for("precision")
    az = synth.insert_azimuths(rng)
    removed = int(rng.integers(8))
    x_warm = synth.part_phantom(s, az)
    x_part = synth.part_phantom(s, az, removed=removed)
    o = oracle.Setup(**s.fields())
    p = oracle.log_transform(synth.poisson_counts(oracle.project(o, x_part), I0,
                                                  np.random.default_rng(POISSON_SEED)), I0)
    w = synth.roi_weights(s)
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(s.n_vox, size=N_SAMPLE, replace=False))
    return s, p, x_warm, w, idx


def stored(a, dtype: str) -> np.ndarray:
    """Values of ``a`` as FP32 then ``dtype`` hold them, widened to FP64 (torch rounds)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    if dtype != "f32":
        t = t.to({"f16": torch.float16, "bf16": torch.bfloat16}[dtype])
    return t.float().numpy().astype(np.float64)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    import oracle
    oracle.build()
    if args.threads:
        oracle.set_num_threads(args.threads)
    path = cache_path()
    if os.path.exists(path):
        print(path, "exists")
        return 0
    s, p, x_warm, w, idx = inputs()
    o = oracle.Setup(**s.fields())
    out = {"idx": idx.astype(np.int64), "p_f32": p.astype(np.float32),
           "settings": np.array(json.dumps(settings(), sort_keys=True, default=str))}
    for dt in DTYPES:
        ps, x = stored(p, dt), stored(x_warm, dt)
        t0 = time.perf_counter()
        for k in range(1, max(SWEEPS) + 1):
            x = oracle.sart(o, ps, x0=x, w=w, n_iter=1, lam=LAMBDA)
            if k in SWEEPS:
                out[f"{dt}_sweep{k}"] = x.reshape(-1)[idx]
                print(f"{dt} sweep {k}: {time.perf_counter() - t0:.0f} s", flush=True)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **out)
    os.replace(tmp, path)
    print(path)
    return 0


if __name__ == "__main__":
    sys.exit(main())
