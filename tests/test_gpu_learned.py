"""GPU tests of the learned-proposal stage against its CPU oracle and the
direct method.

* featurizer, MLP forward and loss/gradient kernels against oracle/learned.py
  (the oracle emulates the kernels' bfloat16 rounding points, so the
  remaining difference is FP32 vs FP64 accumulation): on a dyadic lattice
  of weights and inputs the forward pass is exact on both sides and the
  logits agree bit for bit; every gradient element lies within its own
  rounding bound (tests/learned_bounds.py);
* AdamW against the oracle's update, element by element, over three steps;
* the windowed refine: every proposed window's first maximum against the
  oracle's periodogram over that window's bins, the stop / fallback decision
  replayed from the oracle's window maxima (exactly), and the fallback
  objects' full-grid maximum against the oracle; with every object sent to
  the full grid it returns exactly lsp_batch's peaks; with the true window
  proposed first it finds the full-grid peak;
* training on periodograms of the direct method lowers the loss, and a
  checkpoint resumes bit-exactly;
* ablation: the trained network reaches the same recovery as an untrained
  one while evaluating a fraction of its pairs.
"""
import numpy as np
import pytest

import learned_bounds as LB
import oracle
import synth
from oracle import learned as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2105_04006_gb300 import build
    build.build()
    import paper_2105_04006_gb300 as lsp
    from paper_2105_04006_gb300 import learned as L
    return lsp, L, torch, torch.device("cuda", 0)


def _on_dev(env, b):
    lsp, L, torch, dev = env
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(np.float32), device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    return t, y, off, lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)


def test_featurizer_matches_oracle(env):
    lsp, L, torch, dev = env
    b = synth.ragged_survey(60, seed=5)
    # add an unsorted object and degenerate ones
    rng = np.random.default_rng(2)
    extra_t = [rng.uniform(60000, 60100, 80), np.array([60000.0]), np.array([60000.0, 60001.0, 60002.0])]
    extra_y = [rng.normal(0, 1, 80), np.array([1.0]), np.array([2.0, 2.0, 2.0])]
    t = np.concatenate([b.t] + extra_t)
    y = np.concatenate([b.y] + extra_y)
    off = np.concatenate([b.offsets, b.offsets[-1] + np.cumsum([len(a) for a in extra_t])]).astype(np.int64)
    bb = synth.Batch(t, y, off, b.grid, np.zeros(off.size - 1), np.zeros(off.size - 1))
    td, yd, od, g = _on_dev(env, bb)
    f16, f32 = L.featurize(td, yd, od, g, want_f32=True)
    ref = OL.featurize_batch(bb.t, bb.y.astype(np.float32).astype(np.float64), bb.offsets, g.f_min, g.f_max)
    got = f32.cpu().numpy()
    assert np.max(np.abs(got[:, :256] - ref[:, :256])) <= 1e-4
    assert np.max(np.abs(got[:, 256:] - ref[:, 256:])) <= 1e-5  # exact pair counts
    np.testing.assert_array_equal(f16.float().cpu().numpy(), OL.bf16(got))
    assert not got[-1].any() and not got[-2].any()


def test_forward_matches_oracle(env):
    lsp, L, torch, dev = env
    prop = L.Proposer(100_000, dev, seed=11)
    shapes = OL.layer_shapes(n_classes=prop.dims.n_classes)
    g = np.random.default_rng(3)
    theta = OL.init_params(shapes, seed=11) + g.normal(0, 0.01, prop.n_params)
    prop.params.copy_(torch.tensor(theta, dtype=torch.float32))
    prop.refresh_bf16()
    theta32 = prop.params.cpu().numpy().astype(np.float64)
    x = torch.tensor(g.normal(0, 1, (96, 512)), dtype=torch.float32, device=dev).to(torch.bfloat16)
    lab = torch.tensor(g.integers(0, prop.dims.n_classes, 96), dtype=torch.int32, device=dev)
    xr = x.float().cpu().numpy().astype(np.float64)
    logits = prop.forward(x).cpu().numpy()
    lref, _ = OL.forward(theta32, xr, shapes, bf16_mode=True)
    assert np.max(np.abs(logits - lref)) <= 1e-4 * max(1.0, np.abs(lref).max())
    loss = prop.loss_grad(x, lab).item()
    lo, _ = OL.loss_and_grad(theta32, xr, lab.cpu().numpy(), shapes, bf16_mode=True)
    assert abs(loss - lo) <= 1e-5 * max(1.0, abs(lo))


@pytest.mark.parametrize("seed", [0, 7])
def test_gradient_elementwise_on_dyadic_lattice(env, seed):
    """Forward bit-exact, loss within FP32 rounding, and every gradient element
    (W1, b1, ..., W4, b4) within its rounding bound of the oracle's."""
    lsp, L, torch, dev = env
    prop = L.Proposer(100_000, dev, seed=1)
    shapes = OL.layer_shapes(n_classes=prop.dims.n_classes)
    theta, xv, labv = LB.dyadic_problem(shapes, 96, seed)
    prop.params.copy_(torch.tensor(theta, dtype=torch.float32))
    prop.refresh_bf16()
    assert np.array_equal(prop.params.cpu().numpy().astype(np.float64), theta)  # the lattice is exact in FP32
    x = torch.tensor(xv, dtype=torch.float32, device=dev).to(torch.bfloat16)
    assert np.array_equal(x.float().cpu().numpy().astype(np.float64), xv)  # and in bfloat16
    lab = torch.tensor(labv, dtype=torch.int32, device=dev)
    lo, gref, inter = OL.loss_and_grad(theta, xv, labv, shapes, bf16_mode=True, return_intermediates=True)
    biases = [b for _, b in OL.unpack(theta, shapes)]
    ok, info = LB.lattice_exact(inter, biases)
    assert ok, info  # premise: every forward sum is exact in FP32
    logits = prop.forward(x).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(logits, inter["z"][-1])
    loss = prop.loss_grad(x, lab).item()
    assert abs(loss - lo) <= 1e-6 * max(1.0, abs(lo))
    grad = prop.grad.cpu().numpy().astype(np.float64)
    bound, _ = LB.grad_bound(inter, labv)
    err = np.abs(grad - gref)
    at, worst = 0, []
    for l, (a, b) in enumerate(shapes):
        for name, n in ((f"W{l + 1}", a * b), (f"b{l + 1}", b)):
            r = err[at:at + n] / np.maximum(bound[at:at + n], 1e-300)
            i = int(np.argmax(r))
            worst.append((name, float(r[i]), float(gref[at + i]), float(grad[at + i]), float(bound[at + i])))
            at += n
    assert all(w[1] <= 1.0 for w in worst), worst
    # the bound is tight enough to see a mistake: most elements within 1 % of their size
    nz = gref != 0
    assert np.median(bound[nz] / np.abs(gref[nz])) < 0.01


def test_adamw_matches_oracle(env):
    """Three AdamW steps (decoupled weight decay, bias correction by step) on
    the GPU against the oracle's update, element by element at FP32 rounding
    (a bound of a few ulp per operation, propagated), each step from the GPU's
    own previous state; the bfloat16 copy is the rounding of the FP32
    parameters, bit for bit."""
    lsp, L, torch, dev = env
    prop = L.Proposer(100_000, dev, seed=4)
    n = prop.n_params
    g = np.random.default_rng(12)
    lr, b1, b2, eps, wd = 3e-3, 0.9, 0.999, 1e-8, 0.05
    # the kernel's hyperparameters are FP32: the oracle gets the same values
    f = lambda v: float(np.float32(v))
    for step in range(1, 4):
        grad = g.normal(0, 1e-2, n) * (g.random(n) < 0.9)  # some exact zeros
        grad[:7] = [1e3, -1e3, 1e-30, 0.0, 5.0, -5.0, 1e-6]
        prop.grad.copy_(torch.tensor(grad, dtype=torch.float32))
        p0, m0, v0 = (a.cpu().numpy().astype(np.float64) for a in (prop.params, prop.m, prop.v))
        g32 = prop.grad.cpu().numpy().astype(np.float64)
        lib = lsp.lib()
        import ctypes
        P = ctypes.c_void_p
        assert lib.lsp_mlp_adamw(n, P(prop.params.data_ptr()), P(prop.params16.data_ptr()), P(prop.grad.data_ptr()),
                                 P(prop.m.data_ptr()), P(prop.v.data_ptr()), step, f(lr), f(b1), f(b2), f(eps), f(wd),
                                 None) == 0
        torch.cuda.synchronize()
        p1, m1, v1 = (a.cpu().numpy().astype(np.float64) for a in (prop.params, prop.m, prop.v))
        pr, mr, vr = OL.adamw_step(p0, g32, m0, v0, step, lr=f(lr), beta1=f(b1), beta2=f(b2), eps=f(eps), wd=f(wd))
        u = 2.0 ** -24
        assert np.all(np.abs(m1 - mr) <= 4 * u * (np.abs(f(b1) * m0) + np.abs((1 - f(b1)) * g32)) + 1e-45)
        assert np.all(np.abs(v1 - vr) <= 6 * u * (np.abs(f(b2) * v0) + np.abs((1 - f(b2)) * g32 * g32)) + 1e-45)
        # FP32 rounding propagated: m's error is absolute where its two terms
        # cancel; bias corrections, sqrt, divisions and the update add a few ulp
        c1, c2 = 1 - f(b1) ** step, 1 - f(b2) ** step
        mh, d = mr / c1, np.sqrt(vr / c2) + f(eps)
        am = (np.abs(f(b1) * m0) + np.abs((1 - f(b1)) * g32)) / c1
        tol_upd = (4 * u * am + 8 * u * np.abs(mh)) / d + 2 * u * np.abs(f(wd) * p0)
        tol = 2 * u * np.abs(pr) + f(lr) * tol_upd + 2 * u * f(lr) * (np.abs(mh) / d + np.abs(f(wd) * p0)) + 1e-45
        bad = np.abs(p1 - pr) > tol
        assert not bad.any(), (np.flatnonzero(bad)[:5], p1[bad][:5], pr[bad][:5])
        np.testing.assert_array_equal(prop.params16.float().cpu().numpy().astype(np.float64),
                                      OL.bf16(prop.params.cpu().numpy()))


def test_top_classes(env):
    lsp, L, torch, dev = env
    logits = torch.tensor([[0.0, 3.0, 3.0, 1.0, -2.0], [5.0, 4.0, 3.0, 2.0, 1.0]], device=dev)
    import ctypes
    out = torch.empty((2, 3), dtype=torch.int32, device=dev)
    lib = lsp.lib()
    assert lib.lsp_top_classes(ctypes.c_void_p(logits.data_ptr()), 2, 5, 3, ctypes.c_void_p(out.data_ptr()),
                               None) == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [[1, 2, 3], [0, 1, 2]]


@pytest.fixture(scope="module")
def labelled(env):
    lsp, L, torch, dev = env
    return L.labelled_set(3000, dev, "learned_infer", part=3)


def test_refine_all_fallback_equals_full_grid(env, labelled):
    lsp, L, torch, dev = env
    s = labelled
    n = s["batch"].n_obj
    cls = torch.zeros((n, 2), dtype=torch.int32, device=dev)
    peaks, info = L.refine(s["t"], s["y"], s["off"], s["grid"], cls, 2, 2.0, 2.0)  # nothing stops
    # the refine's own kernel configuration: the same sums, bit for bit
    _, full = lsp.batch(s["t"], s["y"], s["off"], s["grid"], k_reseed=16, freqs_per_thread=32, block_threads=64)
    a, b = lsp.peaks_to_numpy(peaks), lsp.peaks_to_numpy(full)
    np.testing.assert_array_equal(a["idx"], b["idx"])
    np.testing.assert_array_equal(a["power"], b["power"])
    assert ((info.cpu().numpy() & 256) != 0).all()


def test_refine_true_window_first(env, labelled):
    lsp, L, torch, dev = env
    s = labelled
    n = s["batch"].n_obj
    cls = torch.stack([s["labels"], torch.zeros_like(s["labels"])], dim=1).contiguous()
    peaks, info = L.refine(s["t"], s["y"], s["off"], s["grid"], cls, 2, 0.0, 0.0, False)
    got = lsp.peaks_to_numpy(peaks)
    full = s["full_idx"].cpu().numpy()
    assert np.mean(np.abs(got["idx"] - full) <= 1) >= 0.999
    assert ((info.cpu().numpy() & 255) == 1).all()  # stop after the first window


def _pick_threshold(cands, values, margin):
    """The first candidate at least `margin` away from every value (decisions
    taken on either side of it cannot differ between FP32 and FP64 powers)."""
    for c in cands:
        if np.min(np.abs(values - c)) > margin:
            return c
    raise AssertionError("no threshold clear of the window maxima")


def test_refine_windows_match_oracle(env):
    """~200 survey-shaped objects (N_t 50..500, N_f 1e5) with hand-set window
    classes: the true window (from the injected period), wrong windows and the
    two edge windows (moved inside the grid), in four rank orders.

    1. Each window alone (k_windows = 1, stop at once): the refine's first
       maximum against the oracle's periodogram over that window's bins --
       power within 1e-4 at the reported bin and of the oracle's maximum, bin
       within one of it (or a near-tie within 1e-4).
    2. All three windows with stop and fallback thresholds: the number of
       windows evaluated and the fallback flag equal the oracle's replay of the
       refine rule on its own window maxima, exactly; the result matches the
       oracle's best window or, for fallback objects, its full-grid maximum.
    """
    lsp, L, torch, dev = env
    b = synth.learned_set(192, "learned_infer", part=11)
    t, y, off, g = _on_dev(env, b)
    n, n_f = b.n_obj, g.n_f
    n_cls = L.n_classes(n_f)
    k_true = np.floor((b.f_true - g.f_min) / g.df).astype(np.int64)
    true_c = np.clip(k_true // L.STRIDE, 0, n_cls - 1)
    wrong = (true_c + n_cls // 2) % n_cls
    wrong2 = (true_c + n_cls // 3) % n_cls
    edge0, edge1 = np.zeros(n, np.int64), np.full(n, n_cls - 1, np.int64)
    orders = [(true_c, wrong, edge0), (wrong, true_c, edge1), (edge0, edge1, true_c), (wrong, wrong2, edge0)]
    classes = np.stack([np.array([orders[o % 4][r][o] for r in range(3)]) for o in range(n)]).astype(np.int32)
    yseen = b.y.astype(np.float32).astype(np.float64)

    # the oracle's periodogram over each proposed window
    wmax = np.zeros((n, 3))
    wk = np.zeros((n, 3), np.int64)
    wpow = {}
    for o in range(n):
        sl = slice(b.offsets[o], b.offsets[o + 1])
        for r in range(3):
            bins = OL.window_bins(classes[o, r], n_f, L.WINDOW, L.STRIDE)
            pw, fl = oracle.lsp_single(b.t[sl], yseen[sl], g.f_min, g.f_max, n_f, k_sel=bins)
            assert fl == 0
            wpow[o, r] = (bins, pw)
            wmax[o, r], wk[o, r] = OL.first_max(pw, bins)

    # 1. every window on its own
    for r in range(3):
        cls = torch.tensor(classes[:, r:r + 1].copy(), device=dev)
        peaks, info = L.refine(t, y, off, g, cls, 1, 0.0, 0.0, False)
        pk = lsp.peaks_to_numpy(peaks)
        assert (info.cpu().numpy() == 1).all()
        for o in range(n):
            bins, pw = wpow[o, r]
            kg = int(pk["idx"][o])
            assert bins[0] <= kg <= bins[-1], (o, r, kg)
            assert abs(pk["power"][o] - pw[kg - bins[0]]) <= 1e-4, (o, r)
            assert abs(pk["power"][o] - wmax[o, r]) <= 1e-4, (o, r)
            if abs(kg - wk[o, r]) > 1:
                assert pw[kg - bins[0]] >= wmax[o, r] - 1e-4, (o, r, kg, wk[o, r])

    # 2. ranked windows with thresholds clear of every window maximum
    stop = _pick_threshold([0.5, 0.45, 0.55, 0.4, 0.6], wmax.ravel(), 2e-4)
    fb = _pick_threshold([0.3, 0.28, 0.32, 0.25, 0.35], wmax.ravel(), 2e-4)
    cls = torch.tensor(classes, device=dev)
    fell_back = []
    for inconclusive in (False, True):
        peaks, info = L.refine(t, y, off, g, cls, 3, stop, fb, inconclusive)
        pk = lsp.peaks_to_numpy(peaks)
        info = info.cpu().numpy()
        for o in range(n):
            rep = OL.refine_replay([(wmax[o, r], wk[o, r]) for r in range(3)], stop, fb, inconclusive)
            assert info[o] == rep["rounds"] | (L.REFINE_FALLBACK if rep["fallback"] else 0), (o, info[o], rep)
            if rep["fallback"]:
                fell_back.append((o, int(pk["idx"][o]), float(pk["power"][o])))
                continue
            kg = int(pk["idx"][o])
            assert abs(pk["power"][o] - rep["best_p"]) <= 1e-4, (o, rep)
            if abs(kg - rep["best_k"]) > 1:  # a near-tie between windows or within one
                near = [pw[kg - bins[0]] for (bins, pw) in (wpow[o, r] for r in range(rep["rounds"]))
                        if bins[0] <= kg <= bins[-1]]
                assert near and max(near) >= rep["best_p"] - 1e-4, (o, kg, rep)
    # every decision kind occurred
    assert len(fell_back) > 0 and len(fell_back) < 2 * n
    # fallback objects: the full grid's first maximum against the oracle's
    objs = sorted({o for o, _, _ in fell_back})[:60]
    sub = b.subset(objs)
    ref = oracle.lsp_batch(sub.t, sub.y.astype(np.float32).astype(np.float64), sub.offsets, g.f_min, g.f_max, n_f)
    got = {o: (k, p) for o, k, p in fell_back}
    for i, o in enumerate(objs):
        k, p = got[o]
        assert abs(p - ref["arg_pow"][i]) <= 1e-4, (o, p, ref["arg_pow"][i])
        if abs(k - int(ref["arg_idx"][i])) > 1:
            sl = slice(b.offsets[o], b.offsets[o + 1])
            pk2, _ = oracle.lsp_single(b.t[sl], yseen[sl], g.f_min, g.f_max, n_f, k_sel=[k])
            assert pk2[0] >= ref["arg_pow"][i] - 1e-4, (o, k, ref["arg_idx"][i])


def test_propose_refine_one_call_equals_four_calls(env, labelled):
    """lsp_propose_refine (features -> MLP -> top-k -> refine + fallback in one
    C call) against lsp_featurize, lsp_mlp_forward, lsp_top_classes and
    lsp_refine_windows called in turn: classes, peaks and info bit for bit."""
    lsp, L, torch, dev = env
    s = labelled
    n = s["batch"].n_obj
    prop = L.Proposer(s["grid"].n_f, dev, seed=9, k_windows=4, stop_power=0.45)
    for i in range(20):  # a briefly trained network: proposals differ between objects
        sel = slice(128 * i, 128 * (i + 1))
        prop.train_step(s["x16"][sel].contiguous(), s["labels"][sel].contiguous(), lr=3e-3)
    cls_one = torch.empty((n, 4), dtype=torch.int32, device=dev)
    path = L.LearnedPath(prop)
    for _ in range(2):  # a second call reuses the workspace
        pk1, info1 = path(s["t"], s["y"], s["off"], s["grid"], classes_out=cls_one)
    x16 = L.featurize(s["t"], s["y"], s["off"], s["grid"])
    cls = prop.propose(x16, 4)
    pk2, info2 = L.refine(s["t"], s["y"], s["off"], s["grid"], cls, 4, prop.stop_power, prop.fallback_power,
                          prop.inconclusive_fallback)
    torch.cuda.synchronize()
    assert torch.equal(cls_one, cls)
    assert torch.equal(pk1, pk2) and torch.equal(info1, info2)
    assert len(set(map(tuple, cls.cpu().tolist()))) > 5  # the proposal lists differ between objects


def test_window_labels_follow_the_rule(env, labelled):
    lsp, L, torch, dev = env
    s = labelled
    idx = s["full_idx"].cpu().numpy()
    n_cls = L.n_classes(s["grid"].n_f)
    np.testing.assert_array_equal(s["labels"].cpu().numpy(), np.clip(np.maximum(idx, 0) // L.STRIDE, 0, n_cls - 1))
    # an object without a peak (idx -1) gets class 0; one past the last class is clamped
    rec = np.zeros(3, dtype=lsp.PEAK_DTYPE)
    rec["idx"] = [-1, 5000, 10 ** 7]
    pk = torch.from_numpy(rec.view(np.uint8).copy()).to(dev)
    assert L.window_labels(pk, 3, n_cls).cpu().tolist() == [0, 4, n_cls - 1]


def test_training_lowers_loss_and_resumes_exactly(env, tmp_path):
    lsp, L, torch, dev = env
    s = L.labelled_set(4000, dev, "learned_train", part=77)
    p = L.Proposer(s["grid"].n_f, dev, seed=5)
    x, lab = s["x16"], s["labels"]
    g = np.random.default_rng(0)
    sel = [torch.from_numpy(g.choice(x.shape[0], 512, replace=False)).to(dev) for _ in range(60)]
    first = p.loss_grad(x[sel[0]], lab[sel[0]]).item()
    for i in range(30):
        p.train_step(x[sel[i]].contiguous(), lab[sel[i]].contiguous())
    path = str(tmp_path / "ckpt.pt")
    p.save(path)
    for i in range(30, 60):
        p.train_step(x[sel[i]].contiguous(), lab[sel[i]].contiguous())
    q, _ = L.Proposer.load(path, dev)
    for i in range(30, 60):
        q.train_step(x[sel[i]].contiguous(), lab[sel[i]].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(p.params, q.params) and q.step == p.step == 60
    last = p.loss_grad(x[sel[0]], lab[sel[0]]).item()
    assert last < 0.8 * first


def test_trained_network_beats_untrained(env):
    """Ablation: same recovery, far fewer evaluated pairs with the trained network."""
    lsp, L, torch, dev = env
    train = [L.labelled_set(25_000, dev, "learned_train", part=i) for i in range(4)]
    test = L.labelled_set(4000, dev, "learned_infer", part=1)
    untrained = L.Proposer(test["grid"].n_f, dev, seed=9)
    base = L.evaluate(untrained, test)
    trained = L.Proposer(test["grid"].n_f, dev, seed=9)
    L.train(trained, train, epochs=8, batch_size=1024, lr=2e-3)
    res = L.evaluate(trained, test)
    assert res["recovery"] >= 0.99 and base["recovery"] >= 0.99
    assert res["pair_fraction"] < 0.5 * base["pair_fraction"], (res, base)
    assert res["mean_windows"] < base["mean_windows"]


def test_committed_network_meets_the_targets(env):
    """The committed network (weights/proposer_survey.npz, trained on 1e6
    curves by the library's own kernels) on 20000 fresh survey-shaped objects:
    at least 99 % of the full-grid periods recovered (first maximum within one
    bin) while evaluating under a tenth of the full grid's pairs, through the
    one-call path."""
    import os
    lsp, L, torch, dev = env
    path = os.path.join(os.path.dirname(L.__file__), "weights", "proposer_survey.npz")
    prop, meta = L.Proposer.load_npz(path, dev)
    assert "1000000" in meta["trained_on"]
    s = L.labelled_set(20000, dev, "learned_infer", part=7)
    res = L.evaluate(prop, s)
    assert res["recovery"] >= 0.99 and res["pair_fraction"] < 0.1, res
    pk, info = L.propose_and_refine(prop, s["t"], s["y"], s["off"], s["grid"])
    got = lsp.peaks_to_numpy(pk)
    assert np.mean(np.abs(got["idx"] - s["full_idx"].cpu().numpy()) <= 1) >= 0.99
