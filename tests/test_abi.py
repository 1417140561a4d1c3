"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every function that include/lsp.h declares, and validates arguments on the
host (these calls return before anything would be launched)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lsp_mod():
    from paper_2105_04006_gb300 import build
    build.build()
    import paper_2105_04006_gb300 as lsp
    return lsp


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lsp_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lsp_mod):
    names = _declared_functions()
    assert "lsp_batch" in names and "lsp_periodogram" in names and "lsp_argmax_period" in names
    lib = ctypes.CDLL(lsp_mod.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    # and the binding knows all of them
    assert set(names) <= set(lsp_mod.EXPORTS), set(names) - set(lsp_mod.EXPORTS)


def test_library_is_built_for_sm103a(lsp_mod):
    data = open(lsp_mod.LIB_PATH, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_status_strings_and_defaults(lsp_mod):
    L = lsp_mod.lib()
    assert L.lsp_status_string(0) == b"LSP_OK"
    assert b"invalid" in L.lsp_status_string(1)
    o = L.lsp_default_opts()
    assert (o.precision, o.norm, o.center_y, o.top_k) == (0, 1, 1, 1)
    assert L.lsp_version() >= 10000


@pytest.mark.parametrize("grid,err", [
    ((0.0, 1.0, 10), "f_min"),
    ((-1.0, 1.0, 10), "f_min"),
    ((1.0, 1.0, 10), "f_max"),
    ((1.0, 2.0, 0), "n_f"),
    ((1.0, float("inf"), 10), "finite"),
])
def test_grid_validation(lsp_mod, grid, err):
    g = lsp_mod.Grid(*grid)
    with pytest.raises(lsp_mod.LSPError) as ei:
        lsp_mod.workspace_size(1, 100, g, lsp_mod.make_opts())
    assert ei.value.status == 1 and err in str(ei.value)


def test_option_validation(lsp_mod):
    g = lsp_mod.Grid(0.1, 10.0, 1000)
    for bad in (dict(top_k=4), dict(top_k=0), dict(block_threads=48), dict(block_threads=1024)):
        with pytest.raises(lsp_mod.LSPError):
            lsp_mod.workspace_size(5, 100, g, lsp_mod.make_opts(**bad))
    with pytest.raises(lsp_mod.LSPError) as ei:
        lsp_mod.workspace_size(5, 100, g, lsp_mod.make_opts(k_reseed=5))
    assert ei.value.status == 7  # no such kernel variant


def test_workspace_sizes_grow_with_shape(lsp_mod):
    g = lsp_mod.Grid(0.24, 12.0, 100_000)
    o = lsp_mod.make_opts()
    a = lsp_mod.workspace_size(100, 30_000, g, o)
    b = lsp_mod.workspace_size(1000, 300_000, g, o)
    assert 0 < a < b
    assert b % 256 == 0
    # FP64 records are larger; top-3 adds candidate buffers
    assert lsp_mod.workspace_size(1000, 300_000, g, lsp_mod.make_opts(precision="fp64")) > b
    assert lsp_mod.workspace_size(1000, 300_000, g, lsp_mod.make_opts(top_k=3)) > b


def test_call_validation_without_launch(lsp_mod):
    L = lsp_mod.lib()
    g = lsp_mod.Grid(0.1, 10.0, 100)
    o = lsp_mod.make_opts()
    # NULL inputs are rejected before any launch
    st = L.lsp_periodogram(None, None, 10, ctypes.byref(g), ctypes.byref(o), None, None, None, 0, None)
    assert st == 1
    # too-small workspace
    st = L.lsp_periodogram(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, ctypes.byref(g), ctypes.byref(o),
                           None, None, ctypes.c_void_p(1024), 16, None)
    assert st == 4 and b"workspace" in L.lsp_last_error()
    # misaligned workspace
    need = lsp_mod.workspace_size(1, 10, g, o)
    st = L.lsp_periodogram(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, ctypes.byref(g), ctypes.byref(o),
                           None, None, ctypes.c_void_p(1024 + 8), need, None)
    assert st == 4
    # batch without offsets
    st = L.lsp_batch(ctypes.c_void_p(256), ctypes.c_void_p(512), None, 3, 10, ctypes.byref(g), ctypes.byref(o),
                     None, None, None, 0, None)
    assert st == 1
    # empty batch is a no-op
    st = L.lsp_batch(None, None, None, 0, 0, ctypes.byref(g), ctypes.byref(o), None, None, None, 0, None)
    assert st == 0
    # argmax: n_f must match the grid
    st = L.lsp_argmax_period(ctypes.c_void_p(256), 1, 99, ctypes.byref(g), 0, ctypes.c_void_p(512), None)
    assert st == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2105_04006_gb300 as lsp
    monkeypatch.setattr(lsp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lsp, "_lib", None)
    with pytest.raises(lsp.LibraryNotBuilt):
        lsp.lib()


def test_grid_rule_reproduces_table2(lsp_mod):
    """Section 4.3 / Table 2: df = 0.2 pi / T_max (angular), N_f = (f_max - f_min) / df.

    The table prints f in rad/day and df to four digits; T_max follows from
    df, and the library (cycles/day) must return the printed N_f.
    """
    import math
    path = os.path.join(ROOT, "tests", "golden", "table2_grid.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for name, f_min, f_max, df, n_f in rows:
        f_min, f_max, df, n_f = float(f_min), float(f_max), float(df), int(n_f)
        t_max = 0.2 * math.pi / df
        g = lsp_mod.grid_for_span(f_min / (2 * math.pi), f_max / (2 * math.pi), t_max)
        assert g.n_f == n_f, (name, g.n_f, n_f)
    with pytest.raises(lsp_mod.LSPError):
        lsp_mod.grid_for_span(1.0, 2.0, 0.0)


def test_newer_entry_points_validate_without_launch(lsp_mod):
    L = lsp_mod.lib()
    g = lsp_mod.Grid(0.24, 12.0, 1000)
    o = lsp_mod.make_opts()
    P = ctypes.c_void_p
    # generalized periodogram: workspace query, NULL offsets, too-small workspace
    n = ctypes.c_size_t()
    assert L.lsp_workspace_size_gls(10, 1000, ctypes.byref(g), ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value >= lsp_mod.workspace_size(10, 1000, g, o) // 2 and n.value % 256 == 0
    assert L.lsp_batch_gls(P(256), P(512), None, None, 10, 1000, ctypes.byref(g), ctypes.byref(o), None, None,
                           None, 0, None) == 1
    assert L.lsp_batch_gls(P(256), P(512), None, P(768), 10, 1000, ctypes.byref(g), ctypes.byref(o), None, None,
                           P(1024), 16, None) == 4
    # learned stage: parameter count and argument checks
    dims = lsp_mod.MlpDims(512, 256, 3, 98)
    cnt = ctypes.c_int64()
    assert L.lsp_mlp_param_count(ctypes.byref(dims), ctypes.byref(cnt)) == 0
    assert cnt.value == 512 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 98 + 98
    bad = lsp_mod.MlpDims(512, 256, 0, 98)
    assert L.lsp_mlp_param_count(ctypes.byref(bad), ctypes.byref(cnt)) == 1
    assert L.lsp_top_classes(P(256), 4, 10, 17, P(512), None) == 1  # k > 16
    assert L.lsp_featurize(P(256), P(512), P(768), 3, 100, ctypes.byref(g), ctypes.c_float(0.0), P(1024), None,
                           None) == 1  # lag_max must be > 0
    assert L.lsp_refine_windows(P(256), P(512), P(768), 3, 100, ctypes.byref(g), 1, P(1024), 8, 4096, 1024,
                                ctypes.c_float(0.5), ctypes.c_float(0.3), 1, P(2048), None, P(4096), 1 << 20,
                                None) == 1  # window > 2048
    assert L.lsp_refine_windows(P(256), P(512), P(768), 3, 100, ctypes.byref(g), 1, P(1024), 8, 2048, 1024,
                                ctypes.c_float(0.5), ctypes.c_float(0.3), 1, P(2048), None, P(4096), 16,
                                None) == 1  # workspace too small
    # the learned path in one call: proposer and workspace checks
    net = lsp_mod.Proposer(dims, 256, 512, 2048, 1024, 16.0, 8, 0.5, 0.3, 1, 1)
    n = ctypes.c_size_t()
    assert L.lsp_propose_refine_workspace_size(ctypes.byref(net), 3, 100, ctypes.byref(g), ctypes.byref(n)) == 0
    assert n.value % 256 == 0 and n.value >= 3 * 512 * 2
    args = (P(256), P(512), P(768), 3, 100, ctypes.byref(g), P(2048), None, None)
    assert L.lsp_propose_refine(ctypes.byref(net), *args, P(4096), 16, None) == 1  # workspace too small
    for field, value in (("k_windows", 17), ("lag_max", 0.0), ("params", None), ("window", 4096), ("stride", 0)):
        bad_net = lsp_mod.Proposer.from_buffer_copy(net)
        setattr(bad_net, field, value)
        assert L.lsp_propose_refine(ctypes.byref(bad_net), *args, P(4096), 1 << 30, None) == 1, field
    bad_net = lsp_mod.Proposer.from_buffer_copy(net)
    bad_net.dims = lsp_mod.MlpDims(256, 256, 3, 98)
    assert L.lsp_propose_refine(ctypes.byref(bad_net), *args, P(4096), 1 << 30, None) == 1
    assert b"LSP_FEAT_DIM" in L.lsp_last_error()
    assert L.lsp_window_labels(P(256), 3, 0, 98, P(512), None) == 1  # stride must be >= 1
    # tensor-core MLP: a misaligned input is refused before any launch, as is a short wait-test workspace
    x_bad = P(256 + 2)
    assert L.lsp_mlp_forward(ctypes.byref(dims), P(256), P(512), x_bad, 4, P(1024), P(4096), 1 << 30, None) == 1
    assert b"16-byte aligned" in L.lsp_last_error()
    t_out, n_out = ctypes.c_uint32(), ctypes.c_int32()
    assert L.lsp_mlp_gemm_wait_test(P(256), 1024, ctypes.byref(t_out), ctypes.byref(n_out), None) == 1
    # grid rule
    assert lsp_mod.grid_for_span(0.24, 12.0, 3650.0).n_f == round((12.0 - 0.24) / (0.1 / 3650.0))


def test_struct_layouts_match_the_header(lsp_mod, tmp_path):
    # the binding's ctypes structures against a C compiler's view of include/lsp.h
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lsp.h"
#define F(T, m) printf(#T "." #m " %zu\\n", offsetof(T, m))
int main(void) {
  printf("lsp_grid %zu\\nlsp_opts %zu\\nlsp_peak %zu\\nlsp_config %zu\\nlsp_trial %zu\\nlsp_mlp_dims %zu\\n",
         sizeof(lsp_grid), sizeof(lsp_opts), sizeof(lsp_peak), sizeof(lsp_config), sizeof(lsp_trial),
         sizeof(lsp_mlp_dims));
  printf("lsp_proposer %zu\\n", sizeof(lsp_proposer));
  F(lsp_proposer, params); F(lsp_proposer, params_bf16); F(lsp_proposer, window); F(lsp_proposer, stride);
  F(lsp_proposer, lag_max); F(lsp_proposer, k_windows); F(lsp_proposer, stop_power);
  F(lsp_proposer, fallback_power); F(lsp_proposer, inconclusive_fallback); F(lsp_proposer, norm);
  F(lsp_config, packed); F(lsp_config, trig); F(lsp_config, staging);
  F(lsp_trial, ms); F(lsp_trial, max_err); F(lsp_trial, passed); F(lsp_trial, worst_object);
  F(lsp_peak, power); F(lsp_peak, freq); F(lsp_peak, period); F(lsp_peak, flags);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                check=True).stdout.split("\n") if line)
    L = lsp_mod
    assert int(out["lsp_grid"]) == ctypes.sizeof(L.Grid)
    assert int(out["lsp_opts"]) == ctypes.sizeof(L.Opts)
    assert int(out["lsp_config"]) == ctypes.sizeof(L.Config)
    assert int(out["lsp_trial"]) == ctypes.sizeof(L.Trial)
    assert int(out["lsp_mlp_dims"]) == ctypes.sizeof(L.MlpDims)
    assert int(out["lsp_peak"]) == L.PEAK_DTYPE.itemsize
    assert int(out["lsp_proposer"]) == ctypes.sizeof(L.Proposer) == 72
    for name in ("params", "params_bf16", "window", "stride", "lag_max", "k_windows", "stop_power",
                 "fallback_power", "inconclusive_fallback", "norm"):
        assert int(out["lsp_proposer." + name]) == getattr(L.Proposer, name).offset, name
    for name in ("packed", "trig", "staging"):
        assert int(out["lsp_config." + name]) == getattr(L.Config, name).offset
    for name in ("ms", "max_err", "passed", "worst_object"):
        assert int(out["lsp_trial." + name]) == getattr(L.Trial, name).offset
    for name in ("power", "freq", "period", "flags"):
        assert int(out["lsp_peak." + name]) == L.PEAK_DTYPE.fields[name][1]


def test_host_entry_point_checks_buffers_before_any_call(lsp_mod):
    """execute_host hands raw host pointers to the library, which reads or
    writes exactly the plan's sizes: wrong dtypes, lengths, or peaks records
    are refused in Python first (no plan handle or GPU is touched)."""
    import torch
    lsp = lsp_mod
    plan = object.__new__(lsp.Plan)
    plan.opts = lsp.make_opts()
    plan.grid = lsp.Grid(0.1, 1.0, 100)
    plan.n_obj, plan.total_nt, plan._h = 3, 30, None
    t, y = np.zeros(30), np.zeros(30, dtype=np.float32)
    off = np.array([0, 10, 20, 30], dtype=np.int64)
    dev = torch.device("cuda", 0)
    bad_calls = [
        dict(t=np.zeros(29), y=y, offsets=off),                                   # short t
        dict(t=t, y=np.zeros(30), offsets=off),                                   # FP64 y for an FP32 plan
        dict(t=t, y=y, offsets=off[:3]),                                          # short offsets
        dict(t=t, y=y, offsets=None),                                             # batch without offsets
        dict(t=t, y=y, offsets=off, power=np.zeros((3, 99), dtype=np.float32)),    # short power
        dict(t=t, y=y, offsets=off, power=torch.zeros((3, 100), dtype=torch.float64)),  # wrong dtype
        dict(t=t, y=y, offsets=off, peaks=np.empty(2, dtype=lsp.PEAK_DTYPE)),      # too few records
        dict(t=t, y=y, offsets=off, peaks=torch.empty(3 * 40 - 1, dtype=torch.uint8)),
    ]
    for kw in bad_calls:
        with pytest.raises((TypeError, ValueError)):
            plan.execute_host(device=dev, **kw)
