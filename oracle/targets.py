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
                **{"lambda": lam}, alpha=alpha, beta=beta, init_seed=init_seed,
                order="shuffled SGD (binary64), seeds %d.." % order_seed,
                epochs=epochs, test_rmse=rmses,
                seconds_generate=round(t_gen, 1),
                seconds_oracle=round(time.time() - t1, 1))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--config", choices=sorted(CONFIGS), default="netflix")
    ap.add_argument("--scale", type=float, default=0.1)
    ap.add_argument("--epochs", type=int, default=20)
    a = ap.parse_args(argv)
    res = compute(a.config, a.scale, a.epochs)
    allr = load()
    allr[key(a.config, a.scale)] = res
    with open(TARGETS, "w") as f:
        json.dump(allr, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
