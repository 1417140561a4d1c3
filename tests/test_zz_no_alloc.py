"""lsp_batch_noalloc: the batch periodogram for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).

Called through the C ABI twice in a row on the same inputs; each result must
match the regular lsp_batch (caller workspace) within the tolerances of the
other GPU tests -- for a multi-object batch and for one object split over
its observations (whose slices, partial sums and completion counters live in
the shared array and must not carry over from one call to the next).  A
shape too large for the fixed array must be rejected before anything runs,
and an empty batch returns at once.  This file sorts last so that a
stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2105_04006_gb300 import build
    build.build()
    import paper_2105_04006_gb300 as lsp
    return lsp, torch, torch.device("cuda", 0)


def test_noalloc_matches_workspace_entry_point(env):
    lsp, torch, dev = env
    b = synth.ragged_survey(300, seed=41, grid=synth.Grid(0.24, 12.0, 20011))
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    opts = lsp.make_opts(top_k=3)
    assert lsp.workspace_size(b.n_obj, b.t.size, g, opts) <= (32 << 20)
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(np.float32), device=dev)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    ref_power, ref_peaks = lsp.batch(t, y, off, g, top_k=3, return_power=True)
    torch.cuda.synchronize()
    ref_p = ref_power.cpu().numpy()
    ref_k = lsp.peaks_to_numpy(ref_peaks)

    L = lsp.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        power = torch.full((b.n_obj, g.n_f), -1.0, dtype=torch.float32, device=dev)
        peaks = torch.zeros(b.n_obj * 3 * 40, dtype=torch.uint8, device=dev)
        st = L.lsp_batch_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(off.data_ptr()), b.n_obj, b.t.size, ctypes.byref(g),
                                 ctypes.byref(opts), ctypes.c_void_p(power.data_ptr()),
                                 ctypes.c_void_p(peaks.data_ptr()), stream)
        assert st == 0, L.lsp_last_error()
        torch.cuda.synchronize()
        got_p = power.cpu().numpy()
        got_k = lsp.peaks_to_numpy(peaks)
        assert np.max(np.abs(got_p.astype(np.float64) - ref_p)) <= TOL32, call
        assert np.all(np.abs(got_k["idx"] - ref_k["idx"]) <= 1), call
        assert np.max(np.abs(got_k["power"] - ref_k["power"])) <= TOL32, call
        np.testing.assert_array_equal(got_k["flags"], ref_k["flags"])


def test_noalloc_prepare_and_one_split_object(env):
    """One object of 20000 observations on 30011 frequencies, split over six
    slices of observations: two calls in a row against lsp_batch."""
    lsp, torch, dev = env
    L = lsp.lib()
    assert L.lsp_noalloc_prepare() == 0, L.lsp_last_error()
    b = synth.single_small(n_t=20_000, grid=synth.Grid(0.1, 10.0, 30_011))
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    opts = lsp.make_opts(obs_split=6)
    assert lsp.workspace_size(1, b.t.size, g, opts) <= (32 << 20)
    t = torch.tensor(b.t, dtype=torch.float64, device=dev)
    y = torch.tensor(b.y.astype(np.float32), device=dev)
    off = torch.tensor([0, b.t.size], dtype=torch.int64, device=dev)
    ref_power, ref_peaks = lsp.batch(t, y, off, g, return_power=True, obs_split=6)
    torch.cuda.synchronize()
    ref_p = ref_power.cpu().numpy().astype(np.float64)
    ref_k = lsp.peaks_to_numpy(ref_peaks)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        power = torch.full((1, g.n_f), -1.0, dtype=torch.float32, device=dev)
        peaks = torch.zeros(40, dtype=torch.uint8, device=dev)
        st = L.lsp_batch_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(off.data_ptr()), 1, b.t.size, ctypes.byref(g), ctypes.byref(opts),
                                 ctypes.c_void_p(power.data_ptr()), ctypes.c_void_p(peaks.data_ptr()), stream)
        assert st == 0, L.lsp_last_error()
        torch.cuda.synchronize()
        assert np.max(np.abs(power.cpu().numpy().astype(np.float64) - ref_p)) <= TOL32, call
        got_k = lsp.peaks_to_numpy(peaks)
        assert abs(int(got_k["idx"][0]) - int(ref_k["idx"][0])) <= 1, call
        assert abs(got_k["power"][0] - ref_k["power"][0]) <= TOL32, call


def test_noalloc_empty_batch_returns_at_once(env):
    lsp, torch, dev = env
    g = lsp.Grid(0.24, 12.0, 1000)
    opts = lsp.make_opts()
    assert lsp.lib().lsp_batch_noalloc(None, None, None, 0, 0, ctypes.byref(g), ctypes.byref(opts), None, None,
                                       None) == 0


def test_noalloc_rejects_shapes_beyond_its_scratch(env):
    lsp, torch, dev = env
    g = lsp.Grid(0.24, 12.0, 100_000)
    opts = lsp.make_opts()
    n_obj, total = 10_000, 3_000_000  # ~100 MB of scratch
    assert lsp.workspace_size(n_obj, total, g, opts) > (32 << 20)
    L = lsp.lib()
    st = L.lsp_batch_noalloc(ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(1024), n_obj,
                             total, ctypes.byref(g), ctypes.byref(opts), None, None, None)
    assert st == 4
    assert b"static array holds" in L.lsp_last_error()
