"""Learned launch-configuration cost model: data, training and regret.

No counterpart in the paper (auto-tuning is named as future work, §8).  The
workflow, all on the GPU through libjacc.so:

1. timing tables: for (stencil, dtype, side) the exhaustive autotuner
   (`jacc.autotune`) times all 24 tile configurations (median of 5 runs);
2. training: the MLP (`jacc.CostModel`, FP32, 4 -> 3x64 -> 1) is fitted by
   the library's own forward/backward/Adam kernels to ln(time in us) of
   every valid (shape, tile) pair, centred per shape (see `xy`);
3. evaluation on held-out sides: the model picks argmin over the 24 tiles;
   regret = t(pick) / t(best) - 1 against the exhaustive search, compared
   with the method without the model: one fixed default tile (the tile with
   the lowest mean log-time over the training tables) and the library's
   built-in default.

Run the full configuration (about 2000 training timings over 5/7/27-point,
FP32/FP64, sides 256-1024, and 200 held-out shapes):
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
        spr = 4
        r = jacc.autotune(dict(stencil=st, dtype=dt, nx=nx, ny=ny, nz=nz, coeffs=coeffs_for(st)), u0, u1,
                          sweeps_per_rep=spr, reps=reps)
        table.append(dict(stencil=st, dtype=dt, side=side, ms=r["ms"], valid=r["valid"]))
        if log:
            log(f"[{i + 1}/{len(queries)}] {st}pt f{dt} side {side}: best tile {r['best_tile']} {r['best_ms']:.4f} ms")
    return table


def xy(table, centred=True):
    """Feature rows and ln(time in microseconds) targets of every valid (shape, tile).

    centred: subtract each shape's mean log-time over its valid tiles.  The
    argmin over tiles is invariant to a per-shape constant, and without it
    the squared error is dominated by the shape's overall scale (which grows
    with side^3 and dtype) instead of the differences between tiles."""
    X, Y = [], []
    for q in table:
        v = [t for t in range(NUM_TILES) if q["valid"][t]]
        lt = [math.log(q["ms"][t] * 1e3) for t in v]
        c = float(np.mean(lt)) if centred else 0.0
        for t, y in zip(v, lt):
            X.append(jacc.features(q["stencil"], q["side"], q["dtype"], t))
            Y.append(y - c)
    return np.asarray(X, dtype=np.float32), np.asarray(Y, dtype=np.float32)


def query_features(table):
    F = np.zeros((len(table), NUM_TILES, 4), dtype=np.float32)
    V = np.zeros((len(table), NUM_TILES), dtype=np.int32)
    for i, q in enumerate(table):
        for t in range(NUM_TILES):
            F[i, t] = jacc.features(q["stencil"], q["side"], q["dtype"], t)
            V[i, t] = 1 if q["valid"][t] else 0
    return F, V


def fit(model, X, Y, epochs=3000, lr=1e-3):
    import torch
    x = torch.from_numpy(X).cuda()
    y = torch.from_numpy(Y).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = model.train(x, y, epochs, lr)
    torch.cuda.synchronize()
    return float(loss.item()), time.perf_counter() - t0


def default_tile(train_table):
    """The method without the model: one fixed tile, the lowest mean ln(time) over the training tables."""
    s = np.zeros(NUM_TILES)
    c = np.zeros(NUM_TILES)
    for q in train_table:
        for t in range(NUM_TILES):
            if q["valid"][t]:
                s[t] += math.log(q["ms"][t])
                c[t] += 1
    m = np.where(c == len(train_table), s / np.maximum(c, 1), np.inf)
    return int(np.argmin(m))


def regrets(table, picks):
    out = []
    for q, p in zip(table, picks):
        ms = np.asarray(q["ms"])
        best = np.min(ms[np.asarray(q["valid"], dtype=bool)])
        out.append(ms[p] / best - 1.0 if p >= 0 and q["valid"][p] else np.inf)
    return np.asarray(out)


def summary(r):
    r = np.asarray(r)
    return dict(mean=float(np.mean(r)), median=float(np.median(r)), p90=float(np.percentile(r, 90)),
                max=float(np.max(r)), exact_best=float(np.mean(r == 0.0)))


def margin_from_training(model, X, Y):
    """Decision margin: half the model's RMS error on its own training targets."""
    import torch
    pred = model.predict(torch.from_numpy(X).cuda()).cpu().numpy()
    return 0.5 * float(np.sqrt(np.mean((pred - Y) ** 2)))


def library_default_tile(q):
    """The tile jacc_specialize picks with tile_id = -1 and no remembered autotuner pick."""
    jacc.autotune_forget()
    nx, ny, nz = shape_for(q["stencil"], q["side"])
    k = jacc.Kernel(q["stencil"], q["dtype"], nx, ny, nz, coeffs=coeffs_for(q["stencil"]))
    t = k.info()["tile_id"]
    k.release()
    return t


def evaluate(model, train_table, test_table, margin=None):
    import torch
    F, V = query_features(test_table)
    f = torch.from_numpy(F).cuda()
    v = torch.from_numpy(V).cuda()
    model.pick(f, v)  # warm
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pred, pick, gap = model.pick(f, v)
    e1.record()
    torch.cuda.synchronize()
    picks = pick.cpu().numpy()
    dt = default_tile(train_table)
    lib_default = [library_default_tile(q) for q in test_table]
    out = dict(model=summary(regrets(test_table, picks)),
               fixed_default_tile=dict(tile=dt, **summary(regrets(test_table, [dt] * len(test_table)))),
               library_default_tile=summary(regrets(test_table, lib_default)),
               inference_ms_all_queries=e0.elapsed_time(e1), queries=len(test_table))
    # search cost the model saves: the exhaustive tuner times 24 tiles x 6 runs per query
    out["exhaustive_search_ms_per_query"] = float(np.mean([6 * sum(m for m in q["ms"] if math.isfinite(m))
                                                           for q in test_table]))
    # the model as a filter: time only its k best predicted tiles and keep the
    # fastest (the tables hold every tile's timing, so no new runs are needed)
    P = pred.cpu().numpy()
    for kk in (2, 3):
        picks_k, cost = [], []
        for i, q in enumerate(test_table):
            valid = np.asarray(q["valid"], dtype=bool)
            order = [t for t in np.argsort(P[i]) if valid[t]][:kk]
            ms = np.asarray(q["ms"])
            picks_k.append(int(order[int(np.argmin(ms[order]))]))
            cost.append(6 * float(np.sum(ms[order])))
        out[f"model_top{kk}_timed"] = dict(search_ms_per_query=float(np.mean(cost)),
                                           **summary(regrets(test_table, picks_k)))
    if margin is not None:
        # model with its fallback: queries whose top-2 predicted gap is below the
        # margin go to the exhaustive autotuner (regret 0, search cost paid)
        g = gap.cpu().numpy()
        fb = g < margin
        r = regrets(test_table, picks)
        r = np.where(fb, 0.0, r)
        out["model_with_fallback"] = dict(margin=margin, fallback_fraction=float(np.mean(fb)), **summary(r))
    return out, picks


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--train-per-pair", type=int, default=14)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=40000)
    ap.add_argument("--max-side", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--seed", type=int, default=5)
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
    X, Y = xy(train_table)
    model = jacc.CostModel(seed=args.seed)
    loss, t_train = fit(model, X, Y, args.epochs, args.lr)
    margin = margin_from_training(model, X, Y)
    res, _ = evaluate(model, train_table, test_table, margin)
    res.update(train_samples=int(len(Y)), final_train_mse=loss, train_seconds=t_train, collect_seconds=t_collect,
               epochs=args.epochs, lr=args.lr, seed=args.seed, train_sides=tr, heldout_sides=ho)
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(result=res, train_table=train_table, test_table=test_table), f)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
