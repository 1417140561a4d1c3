"""GPU tests of the learned-proposal stage against its CPU oracle and the
direct method.

* featurizer, MLP forward and loss/gradient kernels against oracle/learned.py
  (the oracle emulates the kernels' bfloat16 rounding points, so the
  remaining difference is FP32 vs FP64 accumulation);
* the windowed refine: with every object sent to the full grid it returns
  exactly lsp_batch's peaks; with the true window proposed first it finds
  the full-grid peak;
* training on periodograms of the direct method lowers the loss, and a
  checkpoint resumes bit-exactly;
* ablation: the trained network reaches the same recovery as an untrained
  one while evaluating a fraction of its pairs.
"""
import numpy as np
import pytest

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


def test_forward_and_gradient_match_oracle(env):
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
    grad = prop.grad.cpu().numpy()
    lo, gref = OL.loss_and_grad(theta32, xr, lab.cpu().numpy(), shapes, bf16_mode=True)
    assert abs(loss - lo) <= 1e-5 * max(1.0, abs(lo))
    assert np.linalg.norm(grad - gref) <= 1e-3 * np.linalg.norm(gref)


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
