"""Target test RMSEs for the time-to-target measurement, written by the
oracle alone (test infrastructure: this script calls only `oracle` and the
seeded input generator `synth`); the values go to
`tests/golden/rmse_targets.json`, which the time-to-target leg of the bench
reads as data.

For a workload generated on the CPU from its seed, it runs the binary64
oracle's textbook SGD (Sec. 2.3, a fresh random permutation of Omega per
epoch) from the initial factors of Sec. 5.1 (Philox4x32-10, the library's
default seed 1), with Table 1's hyperparameters. It records the test RMSE
(Sec. 5.1) after every epoch.

    python -m oracle.targets --config netflix --scale 0.1 --epochs 20

Long runs can write to a file of their own (--out) and be merged into the
targets file afterwards (--merge a.json b.json ...).  With --nomad-workers p
the order is the oracle's serial NOMAD with p workers (the GPU's free-run
order up to the itinerary's draws), kept as the entry's "nomad" target:

    python -m oracle.targets --config netflix --scale 1 --epochs 20 \
        --nomad-workers 1216 --out netflix1_nomad.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
TARGETS = os.path.join(os.path.dirname(HERE), "tests", "golden", "rmse_targets.json")

# name: (generator, k, lambda, alpha, beta) -- Table 1's values
CONFIGS = {
    "netflix": ("netflix_shaped", 100, 0.05, 0.012, 0.05),
    "yahoo": ("yahoo_shaped", 100, 1.0, 0.00075, 0.01),
    "hugewiki": ("hugewiki_shaped", 100, 0.01, 0.001, 0.0),
    "hugewiki-flat": ("hugewiki_flat", 100, 0.01, 0.001, 0.0),
    "tiny": ("tiny_planted", 10, 0.05, 0.012, 0.05),
}


def key(config: str, scale: float) -> str:
    return "%s@%g" % (config, scale)


def load() -> dict:
    if not os.path.exists(TARGETS):
        return {}
    with open(TARGETS) as f:
        return json.load(f)


def compute(config: str, scale: float, epochs: int, init_seed: int = 1,
            order_seed: int = 7) -> dict:
    gen, k, lam, alpha, beta = CONFIGS[config]
    fn = getattr(synth, gen)
    t0 = time.time()
    r = fn(device="cpu") if config == "tiny" else fn(scale, device="cpu")
    tr, tc, tv, er, ec, ev = r.numpy()
    t_gen = time.time() - t0
    # binary32 hyperparameters, as the library receives them
    lam32, a32, b32 = (float(np.float32(x)) for x in (lam, alpha, beta))
    W = oracle.init_factor(r.m, k, init_seed, 0)
    H = oracle.init_factor(r.n, k, init_seed, 1)
    rmses = []
    t1 = time.time()
    for e in range(epochs):
        # one epoch at a time, the step size of epoch e (t = e)
        sa = a32 / (1.0 + b32 * e ** 1.5)
        W, H, _ = oracle.shuffled_sgd(tr, tc, tv, W, H, lam32, sa, 0.0, 1,
                                      order_seed + e)
        rmses.append(oracle.rmse(er, ec, ev, W, H))
    return dict(config=config, scale=scale, workload=r.name, m=r.m, n=r.n,
                nnz_train=int(tr.size), nnz_test=int(er.size), k=k,
                fingerprint=r.fingerprint(),
                **{"lambda": lam}, alpha=alpha, beta=beta, init_seed=init_seed,
                order="shuffled SGD (binary64), seeds %d.." % order_seed,
                epochs=epochs, test_rmse=rmses,
                seconds_generate=round(t_gen, 1),
                seconds_oracle=round(time.time() - t1, 1))


def compute_nomad(config: str, scale: float, epochs: int, workers: int, init_seed: int = 1,
                  order_seed: int = 9) -> dict:
    """The binary64 oracle's serial simulation of NOMAD (Alg. 1 with the
    permutation circulation of Sec. 3.4) with `workers` row blocks (the
    ratings-balanced partition), E epochs from the library's initial factors:
    the free-run order the GPU follows, up to the itinerary's random draws."""
    gen, k, lam, alpha, beta = CONFIGS[config]
    fn = getattr(synth, gen)
    r = fn(device="cpu") if config == "tiny" else fn(scale, device="cpu")
    tr, tc, tv, er, ec, ev = r.numpy()
    lam32, a32, b32 = (float(np.float32(x)) for x in (lam, alpha, beta))
    rw = oracle.partition_rows(r.m, tr, workers)
    L = oracle.build_layout(r.m, r.n, tr, tc, tv, rw, workers)
    W = oracle.init_factor(r.m, k, init_seed, 0)
    H = oracle.init_factor(r.n, k, init_seed, 1)
    t1 = time.time()
    W, H, _, _ = oracle.serial_nomad(L, W, H, lam32, a32, b32, epochs, order_seed)
    return dict(config=config, scale=scale, workload=r.name, fingerprint=r.fingerprint(),
                order="serial NOMAD (binary64), %d workers, seed %d" % (workers, order_seed),
                p=workers, epochs=epochs, test_rmse=oracle.rmse(er, ec, ev, W, H),
                seconds_oracle=round(time.time() - t1, 1))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--config", choices=sorted(CONFIGS), default="netflix")
    ap.add_argument("--scale", type=float, default=0.1)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--out", default=None,
                    help="write this one result to a file instead of merging it into "
                         "tests/golden/rmse_targets.json")
    ap.add_argument("--merge", nargs="*", default=None,
                    help="merge result files written with --out into the targets file")
    ap.add_argument("--order-seed", type=int, default=9,
                    help="serial NOMAD: seed of the itinerary draws")
    ap.add_argument("--nomad-workers", type=int, default=0,
                    help="the oracle's serial NOMAD with this many workers instead of "
                         "shuffled SGD (stored as the entry's 'nomad' target)")
    a = ap.parse_args(argv)
    if a.merge is not None:
        allr = load()
        for path in a.merge:
            with open(path) as f:
                res = json.load(f)
            kk = key(res["config"], res["scale"])
            if "p" in res:  # a serial NOMAD target: kept beside the shuffled one
                ent = allr.setdefault(kk, {})
                runs = [x for x in ent.get("nomad", {}).get("runs", [])
                        if x["order"] != res["order"]] + [res]
                vals = [x["test_rmse"] for x in runs]
                ent["nomad"] = dict(p=res["p"], epochs=res["epochs"], runs=runs,
                                    test_rmse=float(np.mean(vals)),
                                    test_rmse_std=float(np.std(vals)) if len(vals) > 1 else 0.0)
            else:
                nomad = allr.get(kk, {}).get("nomad")
                allr[kk] = res
                if nomad:
                    allr[kk]["nomad"] = nomad
        with open(TARGETS, "w") as f:
            json.dump(allr, f, indent=1)
        return
    if a.nomad_workers > 0:
        res = compute_nomad(a.config, a.scale, a.epochs, a.nomad_workers,
                            order_seed=a.order_seed)
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
        print(json.dumps(res))
        return
    res = compute(a.config, a.scale, a.epochs)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    else:
        allr = load()
        allr[key(a.config, a.scale)] = res
        with open(TARGETS, "w") as f:
            json.dump(allr, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
