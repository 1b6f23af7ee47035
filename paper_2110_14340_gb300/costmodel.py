"""Learned launch-configuration cost model: timing runs and the evaluation report.

No counterpart in the paper (auto-tuning is named as future work, §8).  This
module only orchestrates; every step of the method runs in libjacc.so:

1. timing tables: for (stencil, dtype, side) the exhaustive autotuner
   (`jacc.autotune`) times all 24 tile configurations (median of 5 runs);
2. training: `CostModel.fit_tables` (jacc_costmodel_fit_tables) builds the
   features and the per-query centred ln(time in us) targets of every valid
   (query, tile) and fits the MLP (FP32, 4 -> 3x64 -> 1) with the library's
   own forward/backward/Adam kernels;
3. evaluation on held-out sides (jacc_costmodel_evaluate): the model's pick,
   its regret t(pick) / t(best) - 1 against the exhaustive search, the model
   as a filter over its k best-ranked tiles, and the fallback to the
   exhaustive search below a decision margin calibrated on the training
   tables (jacc_costmodel_margin) so that it fires on a stated fraction of
   queries.  The methods without the model: the best single tile over the
   training tables (jacc_costmodel_fixed_tile) and the library's built-in
   size-aware default; their regret also comes from the library
   (jacc_costmodel_regret).

Run the full configuration (about 2000 training timings over 5/7/27-point,
FP32/FP64, sides 256-1024, and 200 held-out shapes), three training seeds:
    python -m paper_2110_14340_gb300.costmodel --out results.json
"""
import argparse
import json
import math
import time

import numpy as np

from . import inputs, jacc

NUM_TILES = jacc.NUM_TILES
PAIRS = [(5, 32), (5, 64), (7, 32), (7, 64), (27, 32), (27, 64)]


def coeffs_for(stencil):
    if stencil == 5:
        return ()
    if stencil == 7:
        return (0.125,)
    return tuple(float(w) for w in inputs.box27_weights())


def shape_for(stencil, side):
    return (side, side, 1) if stencil == 5 else (side, side, side)


def train_sides(lo=256, hi=1024, n=14, step=16):
    """n sides evenly spaced in [lo, hi], rounded to multiples of `step`."""
    return sorted({int(round((lo + (hi - lo) * i / (n - 1)) / step) * step) for i in range(n)})


def heldout_sides(n, exclude, lo=256, hi=1024, seed=5, step=4):
    """n distinct sides in [lo, hi], multiples of `step`, not in `exclude` (seeded)."""
    u = inputs.uniform64(seed, 50 * n)
    out = []
    for x in u:
        s = int(round((lo + (hi - lo) * x) / step) * step)
        if s not in exclude and s not in out and lo <= s <= hi:
            out.append(s)
        if len(out) == n:
            break
    return sorted(out)


class Buffers:
    """Two device fields per dtype, sized for the largest shape; smaller shapes use a prefix."""

    def __init__(self, max_elems, dtypes=(32, 64), device="cuda"):
        import torch
        self.buf = {}
        for dt in dtypes:
            t = torch.float64 if dt == 64 else torch.float32
            a = inputs.uniform_torch(11, max_elems, device, t)
            self.buf[dt] = (a, a.clone())

    def fields(self, dtype, shape):
        nx, ny, nz = shape
        n = nx * ny * nz
        a, b = self.buf[dtype]
        s = (ny, nx) if nz == 1 else (nz, ny, nx)
        return a[:n].view(*s), b[:n].view(*s)


def collect(queries, bufs, reps=5, log=None):
    """queries: [(stencil, dtype, side)] -> list of dict(stencil, dtype, side, ms[24], valid[24])."""
    table = []
    for i, (st, dt, side) in enumerate(queries):
        nx, ny, nz = shape_for(st, side)
        u0, u1 = bufs.fields(dt, (nx, ny, nz))
        # 4-sweep sequences: for FP64 fixed point two of them are the
        # intermediate sweeps that dominate long runs
        r = jacc.autotune(dict(stencil=st, dtype=dt, nx=nx, ny=ny, nz=nz, coeffs=coeffs_for(st)), u0, u1,
                          sweeps_per_rep=4, reps=reps)
        table.append(dict(stencil=st, dtype=dt, side=side, ms=r["ms"], valid=r["valid"]))
        if log:
            log(f"[{i + 1}/{len(queries)}] {st}pt f{dt} side {side}: best tile {r['best_tile']} {r['best_ms']:.4f} ms")
    return table


def summary(r):
    r = np.asarray(r, dtype=np.float64)
    return dict(mean=float(np.mean(r)), median=float(np.median(r)), p90=float(np.percentile(r, 90)),
                max=float(np.max(r)), exact_best=float(np.mean(r == 0.0)))


def library_default_tile(q):
    """The tile jacc_specialize picks with tile_id = -1 and no remembered autotuner pick."""
    jacc.autotune_forget()
    nx, ny, nz = shape_for(q["stencil"], q["side"])
    k = jacc.Kernel(q["stencil"], q["dtype"], nx, ny, nz, coeffs=coeffs_for(q["stencil"]))
    t = k.info()["tile_id"]
    k.release()
    return t


def search_ms(q):
    """Timing cost of the exhaustive search for one query: 24 tiles x (1 warm-up + 5 timed) runs."""
    return 6.0 * sum(m for m, v in zip(q["ms"], q["valid"]) if v)


def baselines(train_table, test_table):
    """Regret of the methods without the model on the held-out tables."""
    ft = jacc.fixed_tile(train_table)
    lib = [library_default_tile(q) for q in test_table]
    return dict(fixed_tile=dict(tile=ft, **summary(jacc.regret(test_table, [ft] * len(test_table)))),
                library_default_tile=summary(jacc.regret(test_table, lib)))


def evaluate(model, train_table, test_table, fallback_fraction=0.25):
    """The model's regret on the held-out tables: argmin pick, filter over its 2 or 3 best-ranked tiles,
    and with a fallback to the exhaustive search calibrated on the training tables."""
    exhaustive = float(np.mean([search_ms(q) for q in test_table]))
    out = dict(queries=len(test_table), exhaustive_search_ms_per_query=exhaustive)
    ev = model.evaluate(test_table, margin=0.0, topk=1)
    out["model"] = summary([e["regret"] for e in ev])
    for k in (2, 3):
        evk = model.evaluate(test_table, margin=0.0, topk=k)
        out[f"model_top{k}_timed"] = dict(search_ms_per_query=6.0 * float(np.mean([e["search_ms_topk"] for e in evk])),
                                          **summary([e["regret_topk"] for e in evk]))
    margin = model.margin(train_table, fallback_fraction)
    evm = model.evaluate(test_table, margin=margin, topk=1)
    fb = np.array([e["fallback"] for e in evm])
    r = np.where(fb, 0.0, [e["regret"] for e in evm])
    out["model_with_fallback"] = dict(margin=margin, calibrated_fraction=fallback_fraction,
                                      fallback_fraction=float(np.mean(fb)),
                                      search_ms_per_query=float(np.mean(fb)) * exhaustive, **summary(r))
    return out, [e["pick"] for e in ev]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--train-per-pair", type=int, default=14)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=40000)
    ap.add_argument("--max-side", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--seeds", default="5,6,7", help="training seeds (comma-separated)")
    ap.add_argument("--fallback-fraction", type=float, default=0.25)
    ap.add_argument("--tables", default=None,
                    help="reuse the timing tables of an earlier --out file instead of collecting them")
    args = ap.parse_args()
    import torch

    from . import build
    build.build()
    jacc.lib()
    tr = train_sides(256, args.max_side, args.train_per_pair)
    per = int(math.ceil(args.heldout / len(PAIRS)))
    ho = heldout_sides(per, set(tr), 256, args.max_side)
    train_q = [(s, d, side) for s, d in PAIRS for side in tr]
    test_q = [(s, d, side) for s, d in PAIRS for side in ho][:args.heldout]
    if args.tables:
        with open(args.tables) as f:
            old = json.load(f)
        train_table, test_table = old["train_table"], old["test_table"]
        t_collect = old["result"].get("collect_seconds")
    else:
        bufs = Buffers(args.max_side ** 3)
        t0 = time.perf_counter()
        train_table = collect(train_q, bufs, log=print)
        test_table = collect(test_q, bufs, log=print)
        t_collect = time.perf_counter() - t0
    res = dict(baselines=baselines(train_table, test_table), seeds={}, collect_seconds=t_collect,
               epochs=args.epochs, lr=args.lr, train_sides=tr, heldout_sides=ho,
               train_samples=int(sum(sum(1 for v in q["valid"] if v) for q in train_table)))
    for seed in [int(x) for x in args.seeds.split(",")]:
        model = jacc.CostModel(seed=seed)
        t0 = time.perf_counter()
        mse = model.fit_tables(train_table, args.epochs, args.lr)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        ev, _ = evaluate(model, train_table, test_table, args.fallback_fraction)
        res["seeds"][str(seed)] = dict(final_train_mse=mse, train_seconds=t_train, **ev)
        model.release()
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(result=res, train_table=train_table, test_table=test_table), f)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
