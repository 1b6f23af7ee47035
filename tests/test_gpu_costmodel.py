"""GPU parity of the learned cost model (forward, gradients, Adam) against the
FP64 oracle, the pick kernel, persistence, the autotuner, and what the trained
network gains over the method without it."""
import math
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
from paper_2110_14340_gb300 import costmodel, inputs, jacc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2110_14340_gb300 import build
    build.build()
    jacc.lib()


def nerr(g, o):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    return float(np.max(np.abs(g - o)) / np.max(np.abs(o)))


def test_library_initialiser_equals_the_published_generator():
    m = jacc.CostModel(seed=5)
    assert np.array_equal(m.params(), inputs.mlp_init(5))
    assert np.all(m.params()[[256 + i for i in range(64)]] == 0.0)  # b1


def test_forward_and_gradient_match_oracle(orc):
    p = inputs.mlp_init(7)
    x, y = inputs.mlp_dataset(3, 203)  # ragged against the 32-sample chunks
    m = jacc.CostModel(init_params=p)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    pred = m.predict(xt).cpu().numpy()
    p64 = p.astype(np.float64)
    assert nerr(pred, orc.mlp_forward(p64, x.astype(np.float64))) <= 1e-5
    loss, g = m.loss_grad(xt, yt)
    lo, go = orc.mlp_loss_grad(p64, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    assert nerr(g.cpu().numpy(), go) <= 1e-4
    # per layer as well, so a small layer cannot hide behind a large one
    for a, b in ((0, 256), (256, 320), (320, 4416), (4416, 4480), (4480, 8576), (8576, 8640), (8640, 8704)):
        assert nerr(g.cpu().numpy()[a:b], go[a:b]) <= 1e-3, (a, b)


def test_adam_step_matches_oracle(orc):
    p = inputs.mlp_init(9)
    x, y = inputs.mlp_dataset(4, 96)
    m = jacc.CostModel(init_params=p)
    m.train(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), epochs=1, lr=1e-3)
    got = m.params().astype(np.float64)
    p64 = p.astype(np.float64)
    _, go = orc.mlp_loss_grad(p64, x.astype(np.float64), y.astype(np.float64))
    want = p64.copy()
    mm = np.zeros_like(want)
    vv = np.zeros_like(want)
    orc.adam_step(want, go, mm, vv, 1, lr=1e-3)
    big = np.abs(go) > 1e-3 * np.max(np.abs(go))
    assert np.max(np.abs((got - p64)[big] - (want - p64)[big])) <= 1e-6
    assert np.max(np.abs(got - p64)) <= 1e-3 * 1.0001  # every step is at most lr


def test_training_reduces_loss_and_pick_is_the_argmin():
    x, y = inputs.mlp_dataset(5, 1024)
    m = jacc.CostModel(seed=5)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    l0, _ = m.loss_grad(xt, yt)
    m.train(xt, yt, epochs=1500, lr=1e-3)
    l1, _ = m.loss_grad(xt, yt)
    assert l1.item() < 0.05 * l0.item()
    rng = np.random.default_rng(0)
    F = rng.uniform(0, 1, (37, 24, 4)).astype(np.float32)
    V = (rng.uniform(0, 1, (37, 24)) > 0.3).astype(np.int32)
    V[5] = 0  # a query with no valid tile
    pred, pick, gap = m.pick(torch.from_numpy(F).cuda(), torch.from_numpy(V).cuda())
    pr = pred.cpu().numpy()
    pk = pick.cpu().numpy()
    for q in range(37):
        if V[q].sum() == 0:
            assert pk[q] == -1
            continue
        vals = np.where(V[q] == 1, pr[q], np.inf)
        assert pk[q] == int(np.argmin(vals))
        s = np.sort(vals)
        if np.isfinite(s[1]):
            assert gap.cpu().numpy()[q] == np.float32(s[1] - s[0])


def test_save_load_roundtrip():
    m = jacc.CostModel(seed=11)
    m.set_range(256.0, 1024.0, 0.01)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.bin")
        m.save(path)
        m2 = jacc.CostModel(seed=1)
        m2.load(path)
        assert np.array_equal(m2.params(), m.params())
        with open(path, "r+b") as f:
            f.write(b"XXXX")
        with pytest.raises(jacc.JaccError):
            m2.load(path)


def test_autotuner_remembers_its_pick():
    nx = ny = nz = 96
    a = torch.rand(nz, ny, nx, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    jacc.autotune_forget()
    args = dict(stencil=7, dtype=64, nx=nx, ny=ny, nz=nz, coeffs=(0.125,))
    r = jacc.autotune(args, a, b, sweeps_per_rep=1, reps=5)
    ms = np.asarray(r["ms"])
    assert all(r["valid"]) and r["best_tile"] == int(np.argmin(ms)) and r["best_ms"] == ms.min()
    k = jacc.Kernel(**args)
    assert k.info()["tile_id"] == r["best_tile"]
    # odd nx: vector tiles are invalid
    c = torch.rand(9, 10, 33, dtype=torch.float64, device="cuda")
    r2 = jacc.autotune(dict(stencil=7, dtype=64, nx=33, ny=10, nz=9, coeffs=(0.125,)), c, torch.empty_like(c), 1, 5)
    assert [bool(v) for v in r2["valid"]] == [jacc.tile_info(t)["vec16"] is False for t in range(24)]
    jacc.autotune_forget()


def test_autotune_tiles_times_only_the_listed_tiles():
    nx = ny = nz = 64
    a = torch.rand(nz, ny, nx, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    jacc.autotune_forget()
    args = dict(stencil=7, dtype=64, nx=nx, ny=ny, nz=nz, coeffs=(0.125,))
    r = jacc.autotune_tiles(args, a, b, [1, 3, 9], sweeps_per_rep=1, reps=3)
    assert [t for t in range(24) if r["valid"][t]] == [1, 3, 9]
    assert all(math.isinf(r["ms"][t]) for t in range(24) if t not in (1, 3, 9))
    assert r["best_tile"] in (1, 3, 9) and r["best_ms"] == min(r["ms"][t] for t in (1, 3, 9))
    assert jacc.Kernel(**args).info()["tile_id"] == r["best_tile"]
    with pytest.raises(jacc.JaccError):
        jacc.autotune_tiles(args, a, b, [24])
    jacc.autotune_forget()


def test_choose_topk_times_the_models_best_ranked_tiles():
    m = jacc.CostModel(seed=5)
    nx = ny = nz = 64
    args = dict(stencil=7, dtype=64, nx=nx, ny=ny, nz=nz, coeffs=(0.125,))
    a = torch.rand(nz, ny, nx, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    feats = torch.tensor([jacc.features(7, float(nx), 64, t) for t in range(24)], dtype=torch.float32,
                         device="cuda").view(1, 24, 4)
    valid = torch.ones(1, 24, dtype=torch.int32, device="cuda")
    pred, _, _ = m.pick(feats, valid)
    top3 = [int(t) for t in np.argsort(pred.cpu().numpy()[0], kind="stable")[:3]]
    jacc.autotune_forget()
    t = m.choose_topk(args, a, b, 3)
    assert t in top3
    assert jacc.Kernel(**args).info()["tile_id"] == t
    jacc.autotune_forget()


def test_choose_falls_back_outside_the_training_range():
    m = jacc.CostModel(seed=5)
    m.set_range(256.0, 512.0, 0.0)
    args = dict(stencil=5, dtype=64, nx=128, ny=128)
    a = torch.rand(128, 128, dtype=torch.float64, device="cuda")
    t, fb = m.choose(args, a, torch.empty_like(a))
    assert fb and 0 <= t < 24
    t2, fb2 = m.choose(dict(stencil=5, dtype=64, nx=300, ny=300))
    assert not fb2 and 0 <= t2 < 24
    assert jacc.Kernel(stencil=5, dtype=64, nx=300, ny=300).info()["tile_id"] == t2
    jacc.autotune_forget()


def _synthetic_tables(seed, nq):
    """Tables of made-up timings (log-normal around a shape trend), some tiles invalid."""
    rng = np.random.default_rng(seed)
    rows = []
    for q in range(nq):
        st = [5, 7, 27][q % 3]
        dt = [32, 64][(q // 3) % 2]
        side = float(rng.integers(64, 1025))
        ms = np.exp(rng.normal(0.0, 0.4, 24)) * (side / 256.0) ** (2 if st == 5 else 3) * (dt / 32)
        valid = (rng.uniform(0, 1, 24) > 0.25).astype(int)
        valid[q % 24] = 1
        rows.append(dict(stencil=st, dtype=dt, side=side, ms=[float(m) for m in ms], valid=[int(v) for v in valid]))
    return rows


def test_fit_tables_trains_on_the_centred_log_targets():
    # the library's pipeline equals training on features and targets built
    # here from the definition: every valid (query, tile), target ln(1000 ms)
    # minus the query's mean over its valid tiles
    tables = _synthetic_tables(21, 30)
    X, Y = [], []
    for q in tables:
        lt = [math.log(q["ms"][t] * 1e3) for t in range(24) if q["valid"][t]]
        mean = sum(lt) / len(lt)
        for t in range(24):
            if q["valid"][t]:
                X.append(jacc.features(q["stencil"], q["side"], q["dtype"], t))
                Y.append(math.log(q["ms"][t] * 1e3) - mean)
    X = np.asarray(X, dtype=np.float32)
    Y = np.asarray(Y, dtype=np.float32)
    a = jacc.CostModel(seed=13)
    b = jacc.CostModel(seed=13)
    mse = a.fit_tables(tables, epochs=70, lr=1e-3)
    loss = b.train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), 70, 1e-3)
    assert np.array_equal(a.params(), b.params())
    assert mse == float(loss.item())


def test_evaluate_matches_the_oracle_forward_and_regret(orc):
    tables = _synthetic_tables(22, 40)
    p = inputs.mlp_init(17)
    m = jacc.CostModel(init_params=p)
    ev = m.evaluate(tables, margin=0.05, topk=3)
    feats = np.array([[jacc.features(q["stencil"], q["side"], q["dtype"], t) for t in range(24)] for q in tables],
                     dtype=np.float64)
    pred = orc.mlp_forward(p.astype(np.float64), feats.reshape(-1, 4)).reshape(len(tables), 24)
    times = np.array([q["ms"] for q in tables])
    valid = np.array([q["valid"] for q in tables], dtype=bool)
    times_inf = np.where(valid, times, np.inf)
    picks = np.array([e["pick"] for e in ev], dtype=np.int32)
    # regret of the library's picks: the oracle's definition on the same table
    want = orc.regret(times_inf, picks)
    assert np.array_equal(np.array([e["regret"] for e in ev]), want)
    for q in range(len(tables)):
        pv = np.where(valid[q], pred[q], np.inf)
        order = np.argsort(pv, kind="stable")
        gap = pv[order[1]] - pv[order[0]]
        assert abs(ev[q]["gap"] - gap) <= 1e-4 * max(1.0, abs(pv[order[0]]))
        assert ev[q]["fallback"] == (ev[q]["gap"] < 0.05)
        if gap > 1e-3:  # FP32 and FP64 predictions agree on a clear argmin
            assert picks[q] == order[0]
            top3 = [t for t in order[:3]]
            if pv[order[3]] - pv[order[2]] > 1e-3:
                assert ev[q]["regret_topk"] == orc.regret(times_inf[q:q + 1], np.array([top3[int(np.argmin(times[q][top3]))]], np.int32))[0]
                assert ev[q]["search_ms_topk"] == pytest.approx(float(np.sum(times[q][top3])), rel=1e-12)


def test_margin_caps_the_fallback_fraction():
    tables = _synthetic_tables(23, 64)
    m = jacc.CostModel(seed=19)
    gaps = np.array([e["gap"] for e in m.evaluate(tables)])
    for f in (0.0, 0.1, 0.25, 0.5, 1.0):
        g = m.margin(tables, f)
        assert np.sum(gaps < g) < max(f * len(tables), 1e-9) or (f == 0.0 and g == 0.0)
        assert g == 0.0 or g in gaps
    with pytest.raises(jacc.JaccError):
        m.margin(tables, 1.5)


GAIN_SEEDS = (5, 6, 7)
# the model's mean regret must be at least 5 points below the best single
# tile's on every seed (measured on this workload: 15-18 points below, the
# best single tile at about 19 %)
GAIN_MARGIN = 0.05


def test_trained_model_gains_over_the_method_without_it():
    # Reduced workload: 2D sides 256-1024, 3D sides 64-256, four stencil/dtype
    # pairs; timings measured here by the exhaustive autotuner.  The methods
    # without the model: the single tile that is best on average over the
    # training tables, and the library's built-in default rule (read off
    # earlier tables of this kind).  Three training seeds.
    pairs = [(5, 64), (7, 32), (7, 64), (27, 32)]
    tr2 = costmodel.train_sides(256, 1024, 8)
    tr3 = costmodel.train_sides(64, 256, 8, step=8)
    ho2 = costmodel.heldout_sides(6, set(tr2), 256, 1024, seed=12)
    ho3 = costmodel.heldout_sides(6, set(tr3), 64, 256, seed=13, step=8)
    q_train = [(s, d, side) for s, d in pairs for side in (tr2 if s == 5 else tr3)]
    q_test = [(s, d, side) for s, d in pairs for side in (ho2 if s == 5 else ho3)]
    bufs = costmodel.Buffers(256 ** 3)
    train_t = costmodel.collect(q_train, bufs)
    test_t = costmodel.collect(q_test, bufs)
    base = costmodel.baselines(train_t, test_t)
    fixed = base["fixed_tile"]["mean"]
    print("cost-model gain test: without the model", base)
    means = []
    for seed in GAIN_SEEDS:
        m = jacc.CostModel(seed=seed)
        mse = m.fit_tables(train_t, epochs=6000, lr=1e-3)
        res, _ = costmodel.evaluate(m, train_t, test_t, fallback_fraction=0.25)
        print(f"seed {seed}: train MSE {mse:.4f}; model {res['model']}; with fallback {res['model_with_fallback']}")
        assert mse < 0.1  # mean squared error of centred ln(time): a fit within ~30 % per tile
        # the model beats the best single tile by a margin on the held-out shapes
        assert res["model"]["mean"] <= fixed - GAIN_MARGIN, (seed, res["model"]["mean"], fixed)
        # the calibrated fallback fires on a minority and never raises the regret
        assert res["model_with_fallback"]["fallback_fraction"] <= 0.5
        assert res["model_with_fallback"]["mean"] <= res["model"]["mean"]
        means.append(res["model"]["mean"])
        m.release()
    assert float(np.mean(means)) <= 0.6 * fixed
