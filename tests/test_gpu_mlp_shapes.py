"""The proposal network's tensor-core GEMMs (tcgen05 + TMA) on shapes that
exercise every edge of their tiling, through the C ABI, against the CPU
oracle (oracle/learned.py, bfloat16 rounding points emulated):

* ragged rows (batch not a multiple of the 128-row tile) and a batch smaller
  than one tile;
* layer widths that are not multiples of 16 (the tile's column count is
  rounded up and the extra columns are zero-filled) and wider than one
  256-column tile;
* an input width that is not a multiple of 8 (the library copies the input
  to a padded pitch before TMA can read it) and K ranges that end inside a
  64-wide slice;
* the weight gradient's K = batch split over several CTAs and summed in a
  fixed order.

On a dyadic lattice every forward sum is exact in FP32, so the logits agree
with the oracle bit for bit; every gradient element lies within its own
rounding bound (tests/learned_bounds.py).  Two calls give identical results,
and no GEMM tile reports a wait that gave up.
"""
import ctypes

import numpy as np
import pytest

import learned_bounds as LB
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
    return lsp, torch, torch.device("cuda", 0)


def _run(env, in_dim, hidden, n_hidden, n_cls, batch, seed):
    lsp, torch, dev = env
    L = lsp.lib()
    dims = lsp.MlpDims(in_dim, hidden, n_hidden, n_cls)
    shapes = OL.layer_shapes(in_dim=in_dim, hidden=hidden, n_hidden=n_hidden, n_classes=n_cls)
    theta, xv, labv = LB.dyadic_problem(shapes, batch, seed)
    cnt = ctypes.c_int64()
    assert L.lsp_mlp_param_count(ctypes.byref(dims), ctypes.byref(cnt)) == 0
    assert cnt.value == theta.size
    s = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    p32 = torch.tensor(theta, dtype=torch.float32, device=dev)
    p16 = torch.empty(theta.size, dtype=torch.bfloat16, device=dev)
    assert L.lsp_to_bf16(ctypes.c_void_p(p32.data_ptr()), ctypes.c_void_p(p16.data_ptr()), theta.size, s) == 0
    x = torch.tensor(xv, dtype=torch.float32, device=dev).to(torch.bfloat16).contiguous()
    lab = torch.tensor(labv, dtype=torch.int32, device=dev)
    nb = ctypes.c_size_t()
    assert L.lsp_mlp_workspace_size(ctypes.byref(dims), batch, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    out = []
    for _ in range(2):
        logits = torch.full((batch, n_cls), -7.0, dtype=torch.float32, device=dev)
        st = L.lsp_mlp_forward(ctypes.byref(dims), ctypes.c_void_p(p32.data_ptr()), ctypes.c_void_p(p16.data_ptr()),
                               ctypes.c_void_p(x.data_ptr()), batch, ctypes.c_void_p(logits.data_ptr()),
                               ctypes.c_void_p(ws.data_ptr()), nb.value, s)
        assert st == 0, L.lsp_last_error()
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        grad = torch.full((theta.size,), 3.0, dtype=torch.float32, device=dev)
        st = L.lsp_mlp_loss_grad(ctypes.byref(dims), ctypes.c_void_p(p32.data_ptr()),
                                 ctypes.c_void_p(p16.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(lab.data_ptr()), batch, ctypes.c_void_p(loss.data_ptr()),
                                 ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(ws.data_ptr()), nb.value, s)
        assert st == 0, L.lsp_last_error()
        torch.cuda.synchronize()
        out.append((logits.cpu().numpy().astype(np.float64), float(loss.item()),
                    grad.cpu().numpy().astype(np.float64)))
    timeouts = ctypes.c_uint32(99)
    assert L.lsp_mlp_gemm_timeouts(ctypes.byref(timeouts)) == 0
    assert timeouts.value == 0
    return shapes, theta, xv, labv, out


@pytest.mark.parametrize("in_dim,hidden,n_hidden,n_cls,batch", [
    (512, 256, 3, 98, 300),    # the survey network's shape, 3 ragged row tiles
    (36, 40, 2, 7, 77),        # input pitch padded, narrow layers, one partial tile
    (512, 320, 2, 98, 1000),   # layers wider than one 256-column tile
    (200, 24, 1, 130, 2100),   # K ending inside a slice, K = batch split over 11 CTAs
])
def test_gemm_shapes_against_oracle(env, in_dim, hidden, n_hidden, n_cls, batch):
    shapes, theta, xv, labv, out = _run(env, in_dim, hidden, n_hidden, n_cls, batch, seed=in_dim + batch)
    (logits, loss, grad), again = out
    np.testing.assert_array_equal(again[0], logits)  # deterministic
    assert again[1] == loss
    np.testing.assert_array_equal(again[2], grad)
    lo, gref, inter = OL.loss_and_grad(theta, xv, labv, shapes, bf16_mode=True, return_intermediates=True)
    biases = [b for _, b in OL.unpack(theta, shapes)]
    ok, info = LB.lattice_exact(inter, biases)
    assert ok, info  # premise: every forward sum is exact in FP32
    np.testing.assert_array_equal(logits, inter["z"][-1])
    assert abs(loss - lo) <= 1e-6 * max(1.0, abs(lo))
    bound, _ = LB.grad_bound(inter, labv)
    err = np.abs(grad - gref)
    at, worst = 0, []
    for l, (a, b) in enumerate(shapes):
        for name, n in ((f"W{l + 1}", a * b), (f"b{l + 1}", b)):
            r = err[at:at + n] / np.maximum(bound[at:at + n], 1e-300)
            i = int(np.argmax(r))
            worst.append((name, float(r[i]), float(gref[at + i]), float(grad[at + i])))
            at += n
    assert all(w[1] <= 1.0 for w in worst), worst


def test_gemm_wait_runs_out_and_the_device_stays_usable(env):
    """A tile whose first operand slice is withheld: its wait gives up after
    about a second, the kernel returns on its own, its outputs are NaN and the
    timeout is counted; the next network call is exact again."""
    lsp, torch, dev = env
    L = lsp.lib()
    ws = torch.empty(65536, dtype=torch.uint8, device=dev)
    timeouts, nans = ctypes.c_uint32(0), ctypes.c_int32(0)
    s = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    st = L.lsp_mlp_gemm_wait_test(ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(timeouts),
                                  ctypes.byref(nans), s)
    assert st == 0, L.lsp_last_error()
    assert timeouts.value == 1 and nans.value == 128 * 16
    shapes, theta, xv, labv, out = _run(env, 36, 40, 2, 7, 77, seed=113)
    _, _, inter = OL.loss_and_grad(theta, xv, labv, shapes, bf16_mode=True, return_intermediates=True)
    np.testing.assert_array_equal(out[0][0], inter["z"][-1])
