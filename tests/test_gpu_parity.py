"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (written here, applied element by element):
  * FP32 path: |P_n(gpu) - P_n(oracle)| <= 1e-4, argmax within one grid bin;
  * FP64 path: |P_n(gpu) - P_n(oracle)| <= 1e-10;
  * integer work (argmax of a stored periodogram, the fused argmax against
    the kernel's own powers, flags) is compared bit-exactly.
Both sides see identical inputs: the oracle gets the FP32 magnitudes the GPU
gets, widened exactly to FP64.  Full-size workloads are checked on sampled
objects or frequencies the oracle computes one by one, plus properties that
hold at any size.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL64 = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2105_04006_gb300 import build
    build.build()
    oracle.build()
    import paper_2105_04006_gb300 as lsp
    return lsp, torch, torch.device("cuda", 0)


def _dev(torch, dev, a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def _y_seen(y, precision):
    return y.astype(np.float32).astype(np.float64) if precision == "fp32" else y.astype(np.float64)


def single(env, b, precision="fp32", **kw):
    lsp, torch, dev = env
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32 if precision == "fp32" else torch.float64)
    power, peaks = lsp.periodogram(t, y, g, precision=precision, **kw)
    torch.cuda.synchronize()
    return power.cpu().numpy().astype(np.float64), lsp.peaks_to_numpy(peaks)


def batch(env, b, precision="fp32", return_power=False, **kw):
    lsp, torch, dev = env
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32 if precision == "fp32" else torch.float64)
    off = _dev(torch, dev, b.offsets, torch.int64)
    power, peaks = lsp.batch(t, y, off, g, precision=precision, return_power=return_power, **kw)
    torch.cuda.synchronize()
    p = power.cpu().numpy().astype(np.float64) if power is not None else None
    return p, lsp.peaks_to_numpy(peaks)


def oracle_single(b, precision, k_sel=None, norm=1):
    g = b.grid
    return oracle.lsp_single(b.t, _y_seen(b.y, precision), g.f_min, g.f_max, g.n_f, norm=norm,
                             k_sel=k_sel)[0]


def oracle_batch(b, precision, **kw):
    g = b.grid
    return oracle.lsp_batch(b.t, _y_seen(b.y, precision), b.offsets, g.f_min, g.f_max, g.n_f, **kw)


def assert_argmax_close(k_gpu, k_orc, p_orc_row=None, tol=TOL32):
    """Argmax within one bin, or (tie-aware) a bin whose oracle power is within tol of the max."""
    if abs(int(k_gpu) - int(k_orc)) <= 1:
        return
    assert p_orc_row is not None and p_orc_row[int(k_gpu)] >= p_orc_row[int(k_orc)] - tol, \
        (k_gpu, k_orc)


# ---------------------------------------------------------------- variants
FP32_VARIANTS = [
    dict(k_reseed=4, freqs_per_thread=8, block_threads=256),
    dict(k_reseed=8, freqs_per_thread=16, block_threads=256),
    dict(k_reseed=16, freqs_per_thread=32, block_threads=256),
    dict(k_reseed=12, freqs_per_thread=24, block_threads=64),
    dict(k_reseed=8, freqs_per_thread=16, block_threads=128),
    dict(k_reseed=4, freqs_per_thread=8, block_threads=64),
    dict(k_reseed=8, freqs_per_thread=8, block_threads=256),
    dict(k_reseed=16, freqs_per_thread=16, block_threads=96),
]
FP64_VARIANTS = [
    dict(k_reseed=4, freqs_per_thread=4, block_threads=128),
    dict(k_reseed=8, freqs_per_thread=8, block_threads=128),
    dict(k_reseed=16, freqs_per_thread=16, block_threads=256),
]


@pytest.fixture(scope="module")
def small_single():
    # 700 observations: three 256-observation tiles with a ragged tail;
    # 12345 frequencies: several chunks with a ragged last chunk.
    b = synth.single_small(n_t=700, grid=synth.Grid(0.1, 10.0, 12345))
    return b, {p: oracle_single(b, p) for p in ("fp32", "fp64")}


@pytest.mark.parametrize("var", FP32_VARIANTS, ids=lambda v: "K{k_reseed}F{freqs_per_thread}T{block_threads}".format(**v))
def test_single_fp32_variants(env, small_single, var):
    b, ref = small_single
    p, pk = single(env, b, "fp32", obs_split=1, **var)
    err = np.max(np.abs(p - ref["fp32"]))
    assert err <= TOL32, err
    assert_argmax_close(pk["idx"][0], np.argmax(ref["fp32"]), ref["fp32"])
    assert abs(pk["power"][0] - ref["fp32"].max()) <= TOL32


@pytest.mark.parametrize("var", FP64_VARIANTS, ids=lambda v: "K{k_reseed}T{block_threads}".format(**v))
def test_single_fp64_variants(env, small_single, var):
    b, ref = small_single
    p, pk = single(env, b, "fp64", obs_split=1, **var)
    err = np.max(np.abs(p - ref["fp64"]))
    assert err <= TOL64, err
    assert pk["idx"][0] == np.argmax(ref["fp64"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("split", [2, 5, 16])
def test_single_split_nt(env, small_single, precision, split):
    b, ref = small_single
    p, pk = single(env, b, precision, obs_split=split)
    err = np.max(np.abs(p - ref[precision]))
    assert err <= (TOL32 if precision == "fp32" else TOL64), err
    assert_argmax_close(pk["idx"][0], np.argmax(ref[precision]), ref[precision])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_single_psd_normalisation(env, small_single, precision):
    b, _ = small_single
    p, _ = single(env, b, precision, norm="psd")
    ref = oracle_single(b, precision, norm=0)
    scale = max(1.0, ref.max())
    assert np.max(np.abs(p - ref)) <= (TOL32 if precision == "fp32" else TOL64) * scale


# --------------------------------------------------------------- batches
@pytest.fixture(scope="module")
def small_batch():
    b = synth.ragged_survey(40, seed=21, grid=synth.Grid(0.24, 12.0, 6007))
    return b, {p: oracle_batch(b, p, top_k=3, return_power=True) for p in ("fp32", "fp64")}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_power_and_argmax(env, small_batch, precision):
    b, ref = small_batch
    p, pk = batch(env, b, precision, return_power=True)
    err = np.max(np.abs(p - ref[precision]["power"]))
    assert err <= (TOL32 if precision == "fp32" else TOL64), err
    for o in range(b.n_obj):
        if precision == "fp64":
            assert pk["idx"][o] == ref["fp64"]["arg_idx"][o]
        else:
            assert_argmax_close(pk["idx"][o], ref["fp32"]["arg_idx"][o], ref["fp32"]["power"][o])
    np.testing.assert_allclose(pk["freq"], b.grid.f_min + pk["idx"] * b.grid.df, rtol=1e-15)
    np.testing.assert_allclose(pk["period"], 1.0 / pk["freq"], rtol=1e-15)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_top3(env, small_batch, precision):
    b, ref = small_batch
    _, pk = batch(env, b, precision, top_k=3)
    pk = pk.reshape(b.n_obj, 3)
    tol = TOL32 if precision == "fp32" else TOL64
    for o in range(b.n_obj):
        pr = ref[precision]["power"][o]
        if precision == "fp64":
            for r in range(3):
                assert int(pk["idx"][o, r]) == int(ref["fp64"]["top_idx"][o, r]), (o, r)
                assert abs(pk["power"][o, r] - ref["fp64"]["top_pow"][o, r]) <= tol
        else:
            _check_top3(pk["idx"][o], pk["power"][o], pr, ref["fp32"]["top_idx"][o], ref["fp32"]["top_pow"][o], o)


def test_batch_top3_every_variant(env, small_batch):
    # top-3 adds a per-CTA candidate buffer in dynamic shared memory; with
    # the largest tiles (K 16, 256 threads) static + dynamic exceed 48 KB
    b, ref = small_batch
    for var in FP32_VARIANTS:
        _, pk = batch(env, b, "fp32", top_k=3, **var)
        pk = pk.reshape(b.n_obj, 3)
        for o in range(b.n_obj):
            _check_top3(pk["idx"][o], pk["power"][o], ref["fp32"]["power"][o], ref["fp32"]["top_idx"][o],
                        ref["fp32"]["top_pow"][o], (str(var), o))


def test_fused_argmax_matches_own_power(env, small_batch):
    # integer decision in the kernel's own precision: bit-exact
    b, _ = small_batch
    for prec in ("fp32", "fp64"):
        p, pk = batch(env, b, prec, return_power=True)
        for o in range(b.n_obj):
            k = int(np.argmax(p[o]))
            assert pk["idx"][o] == k
            assert pk["power"][o] == p[o, k]


TOP3_VARIANTS = FP32_VARIANTS + [
    dict(k_reseed=12, freqs_per_thread=24, block_threads=128),
    dict(k_reseed=8, freqs_per_thread=16, block_threads=64),
    dict(k_reseed=16, freqs_per_thread=32, block_threads=64),
    dict(k_reseed=12, freqs_per_thread=24, block_threads=224),
]


def _own_top3(p, pk, n_obj, what):
    """The fused top-3 against the oracle's local-maximum rule applied to the
    kernel's own powers (the same FP32 values): bit-exact."""
    pk = pk.reshape(n_obj, 3)
    for o in range(n_obj):
        idx, pw = oracle.top_local_maxima(p[o], 3)
        np.testing.assert_array_equal(pk["idx"][o], idx, err_msg=f"{what} object {o}")
        np.testing.assert_array_equal(pk["power"][o], pw, err_msg=f"{what} object {o}")


def test_fused_top3_matches_own_power(env):
    """Top-3 selection (per-thread candidates, warp rounds, the bins at warp
    and chunk boundaries merged by one warp) against the same rule on the
    kernel's stored powers: every FP32 variant, a prime grid so the last
    chunk of each object is ragged, and short objects whose periodograms have
    a local maximum every bin or two."""
    b = synth.ragged_lognormal(48, seed=5, grid=synth.Grid(0.24, 12.0, 20011))
    for var in TOP3_VARIANTS:
        p, pk = batch(env, b, "fp32", return_power=True, top_k=3, **var)
        _own_top3(p, pk, b.n_obj, str(var))
        assert pk["idx"].min() >= 0


@pytest.mark.parametrize("split", [3, 16])
def test_fused_top3_split_single_matches_own_power(env, small_single, split):
    """The split-N_t combine (one bin per thread) selects the top-3 the same way."""
    b, _ = small_single
    p, pk = single(env, b, "fp32", top_k=3, obs_split=split)
    _own_top3(p[None, :], pk, 1, f"split {split}")


def test_fused_top3_gls_matches_own_power(env):
    """The generalized periodogram's kernels share the FP32 epilogue."""
    lsp, torch, dev = env
    b = synth.ragged_lognormal(32, seed=6, grid=synth.Grid(0.24, 12.0, 9001))
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    e = _dev(torch, dev, np.random.default_rng(3).uniform(0.02, 0.3, b.t.size), torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    for var in (dict(k_reseed=8, freqs_per_thread=16, block_threads=64),
                dict(k_reseed=8, freqs_per_thread=16, block_threads=128),
                dict(k_reseed=4, freqs_per_thread=8, block_threads=256)):
        power, peaks = lsp.batch_gls(t, y, e, off, g, return_power=True, top_k=3, **var)
        torch.cuda.synchronize()
        _own_top3(power.cpu().numpy().astype(np.float64), lsp.peaks_to_numpy(peaks), b.n_obj, str(var))


def test_batch_variants_agree(env, small_batch):
    b, ref = small_batch
    for var in FP32_VARIANTS:
        _, pk = batch(env, b, "fp32", **var)
        for o in range(b.n_obj):
            assert_argmax_close(pk["idx"][o], ref["fp32"]["arg_idx"][o], ref["fp32"]["power"][o])
            assert abs(pk["power"][o] - ref["fp32"]["arg_pow"][o]) <= TOL32


# ------------------------------------------------------------ edge cases
def _custom_batch(segs, grid):
    ts = [np.asarray(s[0], dtype=np.float64) for s in segs]
    ys = [np.asarray(s[1], dtype=np.float64) for s in segs]
    off = np.concatenate([[0], np.cumsum([len(x) for x in ts])]).astype(np.int64)
    t = np.concatenate(ts) if ts else np.zeros(0)
    y = np.concatenate(ys) if ys else np.zeros(0)
    return synth.Batch(t, y, off, grid, np.zeros(len(segs)), np.zeros(len(segs)))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_edge_cases(env, precision):
    lsp = env[0]
    g = synth.Grid(0.24, 12.0, 777)
    rng = np.random.default_rng(5)
    segs = [
        ([], []),                                             # empty
        ([60000.0], [1.0]),                                   # one observation
        ([60000.0, 60001.3], [0.5, -0.2]),                    # two
        ([60000.0, 60001.3, 60007.9], [0.1, 0.7, -0.3]),      # three
        ([60000.0, 60003.0, 60009.0], [2.0, 2.0, 2.0]),       # zero variance
        ([60000.0, 60001.0, 60002.0], [1.0, np.nan, 0.0]),    # NaN
        (np.sort(rng.uniform(60000, 61000, 300)), rng.normal(0, 1, 300)),  # a normal one
        (rng.uniform(60000, 61000, 50)[::-1], rng.normal(0, 1, 50)),     # unsorted times
    ]
    b = _custom_batch(segs, g)
    p, pk = batch(env, b, precision, return_power=True)
    ref = oracle_batch(b, precision, return_power=True)
    np.testing.assert_array_equal(pk["flags"], ref["flags"])
    tol = TOL32 if precision == "fp32" else TOL64
    assert np.max(np.abs(p - ref["power"])) <= tol
    for o in range(b.n_obj):
        if ref["flags"][o]:
            assert pk["idx"][o] == -1 and pk["power"][o] == 0.0
        else:
            assert_argmax_close(pk["idx"][o], ref["arg_idx"][o], ref["power"][o], tol)
    assert pk["flags"][1] & lsp.FLAG_FEW_OBS and pk["flags"][4] & lsp.FLAG_ZERO_VAR
    assert pk["flags"][5] & lsp.FLAG_NONFINITE


def _nightly_batch(n_obj, seed, grid):
    # observations inside a one-hour window of each night: near multiples of
    # 1/2 c/d all doubled phases align and Eq. 2's sin^2 denominator nearly
    # vanishes (the FP32 kernels re-evaluate those bins in FP64)
    rng = np.random.default_rng(seed)
    segs = []
    for _ in range(n_obj):
        n = int(rng.integers(20, 400))
        nights = np.sort(rng.choice(3000, n, replace=False)).astype(np.float64)
        t = 60000.0 + nights + 0.3 + rng.uniform(0, 1.0 / 24.0, n)
        y = 0.4 * np.sin(2 * np.pi * rng.uniform(0.3, 5.0) * t) + rng.normal(0, 0.2, n)
        segs.append((t, y))
    return _custom_batch(segs, grid)


def test_nightly_cadence_ill_conditioned_bins(env):
    b = _nightly_batch(12, 17, synth.Grid(0.24, 12.0, 20011))
    p, pk = batch(env, b, "fp32", return_power=True)
    ref = oracle_batch(b, "fp32", return_power=True)
    assert np.max(np.abs(p - ref["power"])) <= TOL32
    for o in range(b.n_obj):
        assert_argmax_close(pk["idx"][o], ref["arg_idx"][o], ref["power"][o])
    # the same through the split-N_t single-object path (combine kernel)
    one = b.subset([int(np.argmax(b.n_t))])
    p1, _ = single(env, one, "fp32", obs_split=7)
    assert np.max(np.abs(p1 - oracle_single(one, "fp32"))) <= TOL32


def test_one_frequency_and_bad_offsets(env):
    lsp, torch, dev = env
    b = synth.ragged_survey(5, seed=8, grid=synth.Grid(0.5, 0.6, 1))
    p, pk = batch(env, b, "fp64", return_power=True)
    ref = oracle_batch(b, "fp64", return_power=True)
    assert np.max(np.abs(p - ref["power"])) <= TOL64
    assert (pk["idx"] == 0).all()
    # offsets that run backwards / past the end flag the objects they touch
    bad = b.offsets.copy()
    bad[2], bad[3] = bad[3], bad[2]
    bad[5] = bad[5] + 7
    g = lsp.Grid(0.5, 0.6, 1)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, bad, torch.int64)
    _, peaks = lsp.batch(t, y, off, g)
    got = lsp.peaks_to_numpy(peaks)
    assert got["flags"][2] & lsp.FLAG_BAD_OFFSETS and got["flags"][4] & lsp.FLAG_BAD_OFFSETS
    assert got["flags"][0] == 0 and got["idx"][0] == 0


def test_many_frequencies_few_observations(env):
    # a long grid (2^25 bins) for a short light curve: sampled oracle check
    b = synth.single_small(n_t=16, grid=synth.Grid(0.1, 50.0, 1 << 25))
    p, pk = single(env, b, "fp32")
    ks = np.unique(np.concatenate([np.linspace(0, b.grid.n_f - 1, 200).astype(np.int64),
                                   np.arange(-3, 4) + int(pk["idx"][0])]))
    ks = ks[(ks >= 0) & (ks < b.grid.n_f)]
    ref = oracle_single(b, "fp32", k_sel=ks)
    assert np.max(np.abs(p[ks] - ref)) <= TOL32
    assert p.min() >= 0.0 and p.max() <= 1.0 + 1e-5


# ----------------------------------------------------- argmax, exactness
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_argmax_period_exact(env, dtype):
    lsp, torch, dev = env
    rng = np.random.default_rng(1)
    n_obj, n_f = 7, 50_001
    p = rng.integers(0, 50, (n_obj, n_f)).astype(dtype)  # many ties
    p[2, :] = np.nan
    p[3, ::3] = np.nan
    p[4, :] = -1.0
    p[5, 40_000] = 1e30
    g = lsp.Grid(0.3, 9.0, n_f)
    peaks = lsp.peaks_to_numpy(lsp.argmax_period(_dev(torch, dev, p, torch.float32 if dtype == np.float32 else torch.float64), g))
    for o in range(n_obj):
        row = p[o].astype(np.float64)
        if np.all(np.isnan(row)):
            assert peaks["idx"][o] == -1
            continue
        k = int(np.nanargmax(row))  # first maximum among non-NaN
        assert peaks["idx"][o] == k
        assert peaks["power"][o] == row[k]
        assert peaks["freq"][o] == 0.3 + k * ((9.0 - 0.3) / n_f)


def test_determinism_graph_and_host_entry(env, small_batch):
    lsp, torch, dev = env
    b, ref = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    _, pk1 = lsp.batch(t, y, off, g, top_k=3)
    _, pk2 = lsp.batch(t, y, off, g, top_k=3)
    plan = lsp.Plan(b.n_obj, b.t.size, g, top_k=3)
    pk3 = plan.execute(t, y, off)   # captures the graph
    pk4 = plan.execute(t, y, off)   # replays it
    torch.cuda.synchronize()
    a = [lsp.peaks_to_numpy(x) for x in (pk1, pk2, pk3, pk4)]
    for x in a[1:]:
        assert x.tobytes() == a[0].tobytes()
    host = plan.execute_host(b.t, b.y.astype(np.float32), b.offsets)
    assert host.tobytes() == a[0].tobytes()
    plan.close()


def test_autotune_keeps_parity(env, small_batch, tmp_path):
    lsp, torch, dev = env
    b, ref = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    cache = str(tmp_path / "tune.jsonl")
    cfg = plan.autotune(t, y, off, cache_path=cache)
    assert cfg["k_reseed"] in (4, 8, 12, 16)
    pk = lsp.peaks_to_numpy(plan.execute(t, y, off))
    for o in range(b.n_obj):
        assert_argmax_close(pk["idx"][o], ref["fp32"]["arg_idx"][o], ref["fp32"]["power"][o])
    # a second plan reads the cached choice
    plan2 = lsp.Plan(b.n_obj, b.t.size, g)
    assert plan2.autotune(t, y, off, cache_path=cache) == cfg
    plan.close()
    plan2.close()


# ------------------------------------------------------- full-size shapes
def test_autotune_gate_checks_more_than_the_first_object(env):
    """A benign first object (40 observations, a strong sinusoid) before a long
    one (8000 observations: the longest FP32 sums) and an ill-conditioned one
    (one hour per night: at twice the frequency of whole cycles per day every
    phase aligns and N - R is small).  The gate checks all three; the error it
    reports for each equals what the chosen configuration gives against the
    FP64 path on the whole batch; and the largest, which decides the gate, is
    the ill-conditioned object's, above the first object's."""
    lsp, torch, dev = env
    rng = np.random.default_rng(5)
    grid = synth.Grid(0.24, 12.0, 20011)
    t0 = np.sort(rng.uniform(60000, 60400, 40))
    t1 = np.sort(rng.uniform(60000, 63650, 8000))
    t2 = np.sort(60000.0 + rng.choice(3650, 300, replace=False) + rng.uniform(0, 1 / 24, 300))
    segs = [(t0, np.sin(2 * np.pi * 1.7 * t0) + 0.01 * rng.normal(size=40)),
            (t1, rng.normal(0, 1, 8000)),
            (t2, np.sin(2 * np.pi * 0.3 * t2) + 0.2 * rng.normal(size=300))]
    sv = synth.ragged_survey(9, seed=31, grid=grid)
    for o in range(sv.n_obj):
        sl = slice(sv.offsets[o], sv.offsets[o + 1])
        segs.append((sv.t[sl], sv.y[sl]))
    b = _custom_batch(segs, grid)
    g = lsp.Grid(grid.f_min, grid.f_max, grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    cfg, trials = plan.autotune(t, y, off, return_trials=True)
    rep = dict(plan.gate_report())
    assert {0, 1, 2} <= set(rep), rep  # first, longest, worst-conditioned
    assert len(rep) <= 8
    kw = dict(k_reseed=cfg["k_reseed"], freqs_per_thread=cfg["freqs_per_thread"], block_threads=cfg["block_threads"])
    p32, _ = batch(env, b, "fp32", return_power=True, **kw)
    # the FP64 path on the magnitudes the FP32 path sees (FP32, widened)
    b32 = synth.Batch(b.t, b.y.astype(np.float32).astype(np.float64), b.offsets, b.grid, b.f_true, b.sigma)
    p64, _ = batch(env, b32, "fp64", return_power=True)
    for o, e in rep.items():
        assert np.float32(np.max(np.abs(p32[o] - p64[o]))) == np.float32(e), (o, e)
    # the ill-conditioned object, not the first one, sets the gate's error
    assert rep[2] > rep[0] and max(rep, key=rep.get) == 2, rep
    chosen = [tr for tr in trials if tr["passed"] and tr["config"] == cfg]
    assert chosen and chosen[0]["max_err"] == np.float32(max(rep.values()))
    assert chosen[0]["worst_object"] == 2
    plan.close()


def test_full_single_small(env):
    """One object, N_t=1000, N_f=1e5: the full periodogram against the full oracle."""
    b = synth.single_small()
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        p, pk = single(env, b, prec)
        ref = oracle_single(b, prec)
        assert np.max(np.abs(p - ref)) <= tol
        assert_argmax_close(pk["idx"][0], np.argmax(ref), ref, tol)


def _argmax_rates(pk_idx, pk_pow, b, objs, ref):
    """Strict (|dk| <= 1) and tie-aware rates of the GPU's first maxima against
    the oracle's on `objs`; tie-aware: a farther bin passes when the oracle's
    own power there is within 1e-4 of its maximum.  Also the largest peak-power
    error (GPU power against the oracle's at the GPU's bin)."""
    strict, tie, worst = 0, 0, 0.0
    g = b.grid
    y = b.y.astype(np.float32).astype(np.float64)
    for i, o in enumerate(objs):
        kg, ko = int(pk_idx[o]), int(ref["arg_idx"][i])
        if abs(kg - ko) <= 1:
            strict += 1
            tie += 1
            if kg == ko:
                worst = max(worst, abs(pk_pow[o] - ref["arg_pow"][i]))
                continue
        sl = slice(b.offsets[o], b.offsets[o + 1])
        p, _ = oracle.lsp_single(b.t[sl], y[sl], g.f_min, g.f_max, g.n_f, k_sel=[kg])
        worst = max(worst, abs(pk_pow[o] - p[0]))
        if abs(kg - ko) > 1 and p[0] >= ref["arg_pow"][i] - TOL32:
            tie += 1
    n = len(objs)
    return strict / n, tie / n, worst


def test_full_ragged_survey_sampled(env):
    """10000 objects, N_t in [50, 500], N_f=1e5, argmax only (the benchmark's
    launch).  The FP32 first maxima against the FP64 oracle on 1000 objects
    evenly spaced over the batch: at least 99.9 % within one bin, all of them
    tie-aware, peak powers within 1e-4.  Over the whole batch, against the
    FP64 GPU path (itself within 1e-10 of the oracle in the other tests): the
    same 99.9 % and 1e-4."""
    lsp, torch, dev = env
    b = synth.ragged_survey()
    _, pk = batch(env, b, "fp32")
    assert (pk["flags"] == 0).all()
    sample = np.linspace(0, b.n_obj - 1, 1000).astype(np.int64)
    ref = oracle_batch(b.subset(sample), "fp32")
    strict, tie, worst = _argmax_rates(pk["idx"], pk["power"], b, sample, ref)
    assert strict >= 0.999 and tie == 1.0, (strict, tie)
    assert worst <= TOL32, worst
    assert (pk["power"] >= 0).all() and (pk["power"] <= 1.0 + 1e-5).all()
    _, pk64 = batch(env, b, "fp64")
    dk = np.abs(pk["idx"] - pk64["idx"])
    assert np.mean(dk <= 1) >= 0.999, np.mean(dk <= 1)
    same = dk == 0
    assert np.max(np.abs(pk["power"][same] - pk64["power"][same])) <= TOL32


def test_full_single_large_sampled(env):
    """One object, N_t=1e5, N_f=1e6, full periodogram: FP32 and FP64 paths."""
    b = synth.single_large()
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        p, pk = single(env, b, prec)
        k_top = int(pk["idx"][0])
        ks = np.unique(np.concatenate([np.linspace(0, b.grid.n_f - 1, 160).astype(np.int64),
                                       k_top + np.arange(-20, 21)]))
        ks = ks[(ks >= 0) & (ks < b.grid.n_f)]
        ref = oracle_single(b, prec, k_sel=ks)
        assert np.max(np.abs(p[ks] - ref)) <= tol, (prec, np.max(np.abs(p[ks] - ref)))
        assert p.min() >= 0.0 and p.max() <= 1.0 + (1e-5 if prec == "fp32" else 1e-12)
        assert int(np.argmax(p)) == k_top
        # the injected dominant frequency is found within one bin
        assert abs(k_top - (b.f_true[0] - b.grid.f_min) / b.grid.df) <= 1.0


def _check_top3(pk_idx, pk_pow, pr, top_idx, top_pow, what):
    """Top-3 local maxima against the oracle's: where the bins agree the powers
    agree within 1e-4; the GPU's power at its own bin is always within 1e-4 of
    the oracle's there; a different bin is allowed only for a near-tie of two
    local maxima, i.e. oracle powers within the two FP32 errors (2e-4)."""
    for r in range(3):
        kg, ko = int(pk_idx[r]), int(top_idx[r])
        assert abs(pk_pow[r] - pr[kg]) <= TOL32, (what, r, kg)
        if kg == ko:
            assert abs(pk_pow[r] - top_pow[r]) <= TOL32, (what, r)
        else:
            assert abs(pr[kg] - pr[ko]) <= 2 * TOL32, (what, r, kg, ko)


def test_full_ragged_lognormal_top3_sampled(env):
    """100000 objects, N_t log-uniform in [10, 2000], N_f=5e4, argmax + top-3.
    300 objects against the FP64 oracle: 200 evenly spaced and the 100 with
    the most observations (N_t near 2000).  First maxima: at least 99.9 %
    within one bin, all tie-aware; top-3 as in _check_top3."""
    b = synth.ragged_lognormal()
    _, pk = batch(env, b, "fp32", top_k=3)
    pk = pk.reshape(b.n_obj, 3)
    longest = np.argsort(b.n_t, kind="stable")[-100:]
    sample = np.unique(np.concatenate([np.linspace(0, b.n_obj - 1, 200).astype(np.int64), longest]))
    assert sample.size >= 290 and b.n_t[sample].max() >= 1990
    sb = b.subset(sample)
    ref = oracle_batch(sb, "fp32", top_k=3, return_power=True)
    strict = 0
    for i, o in enumerate(sample):
        pr = ref["power"][i]
        kg, ko = int(pk["idx"][o, 0]), int(ref["arg_idx"][i])
        strict += abs(kg - ko) <= 1
        assert abs(kg - ko) <= 1 or pr[kg] >= pr[ko] - TOL32, (o, kg, ko)
        _check_top3(pk["idx"][o], pk["power"][o], pr, ref["top_idx"][i], ref["top_pow"][i], int(o))
    assert strict / sample.size >= 0.999, strict / sample.size


def test_periodogram_written_to_pinned_host_memory(env, small_batch):
    """power_out in page-locked host memory: the kernels write it directly (Section 3.5's return)."""
    lsp, torch, dev = env
    b, ref = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    p_dev, pk_dev = lsp.batch(t, y, off, g, return_power=True)
    host = torch.empty((b.n_obj, g.n_f), dtype=torch.float32).pin_memory()
    host.fill_(-1.0)
    opts = lsp.make_opts()
    ws = torch.empty(lsp.workspace_size(b.n_obj, b.t.size, g, opts), dtype=torch.uint8, device=dev)
    peaks = torch.empty(b.n_obj * 40, dtype=torch.uint8, device=dev)
    import ctypes
    st = lsp.lib().lsp_batch(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                             ctypes.c_void_p(off.data_ptr()), b.n_obj, b.t.size, ctypes.byref(g), ctypes.byref(opts),
                             ctypes.c_void_p(host.data_ptr()), ctypes.c_void_p(peaks.data_ptr()),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                             ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert torch.equal(host, p_dev.cpu())
    # the host entry point takes the same zero-copy route for a pinned power_out
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    host2 = torch.full((b.n_obj, g.n_f), -1.0, dtype=torch.float32).pin_memory()
    pk = plan.execute_host(b.t, b.y.astype(np.float32), b.offsets, power=host2)
    assert torch.equal(host2, p_dev.cpu())
    assert (pk["idx"] == lsp.peaks_to_numpy(pk_dev)["idx"]).all()
    # and the staged route for pageable memory
    host3 = np.full((b.n_obj, g.n_f), -1.0, dtype=np.float32)
    plan.execute_host(b.t, b.y.astype(np.float32), b.offsets, power=host3)
    np.testing.assert_array_equal(host3, p_dev.cpu().numpy())
    plan.close()


@pytest.mark.parametrize("parts", [2, 3, 7])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_periodogram_returned_in_object_groups(env, small_batch, precision, parts):
    """The host entry point's grouped return (copies of one group's rows overlap
    the next groups' kernels, Section 3.5): the same powers and peaks as one
    pass, bit for bit, into pageable and page-locked power_out; 40 objects in
    2, 3 or 7 groups of unequal observation counts."""
    lsp, torch, dev = env
    b, ref = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    ydt = np.float32 if precision == "fp32" else np.float64
    tdt = torch.float32 if precision == "fp32" else torch.float64
    yh = b.y.astype(ydt)
    plan = lsp.Plan(b.n_obj, b.t.size, g, precision=precision, top_k=3)
    plan.set_host_parts(1)
    assert plan.host_parts() == 1
    one = np.full((b.n_obj, g.n_f), -1.0, dtype=ydt)
    pk1 = plan.execute_host(b.t, yh, b.offsets, power=one)
    err = np.max(np.abs(one.astype(np.float64) - ref[precision]["power"]))
    assert err <= (TOL32 if precision == "fp32" else TOL64), err
    plan.set_host_parts(parts)
    assert plan.host_parts() == parts
    pag = np.full((b.n_obj, g.n_f), -1.0, dtype=ydt)
    pk2 = plan.execute_host(b.t, yh, b.offsets, power=pag)
    pin = torch.full((b.n_obj, g.n_f), -1.0, dtype=tdt).pin_memory()
    pk3 = plan.execute_host(b.t, yh, b.offsets, power=pin)
    np.testing.assert_array_equal(pag, one)
    np.testing.assert_array_equal(pin.numpy(), one)
    for pk in (pk2, pk3):
        for name in lsp.PEAK_DTYPE.names:
            np.testing.assert_array_equal(pk[name], pk1[name], err_msg=name)
    # the graph-replayed device path still agrees after the grouped calls
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, yh, tdt)
    off = _dev(torch, dev, b.offsets, torch.int64)
    p_dev = torch.empty((b.n_obj, g.n_f), dtype=tdt, device=dev)
    plan.execute(t, y, off, power=p_dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(p_dev.cpu().numpy(), one)
    plan.close()


def test_host_groups_with_bad_offsets_take_one_pass(env):
    """Offsets that run backwards or past the inputs: the grouped return falls
    back to one pass, which flags the objects they touch (no group reads past
    the inputs)."""
    lsp, torch, dev = env
    b = synth.ragged_survey(8, seed=8, grid=synth.Grid(0.5, 2.0, 301))
    bad = b.offsets.copy()
    bad[2], bad[3] = bad[3], bad[2]
    bad[8] = bad[8] + 7
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    yh = b.y.astype(np.float32)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    one = np.full((b.n_obj, g.n_f), -1.0, dtype=np.float32)
    plan.set_host_parts(1)
    pk1 = plan.execute_host(b.t, yh, bad, power=one)
    grp = np.full((b.n_obj, g.n_f), -1.0, dtype=np.float32)
    plan.set_host_parts(4)
    pk2 = plan.execute_host(b.t, yh, bad, power=grp)
    np.testing.assert_array_equal(grp, one)
    for name in lsp.PEAK_DTYPE.names:
        np.testing.assert_array_equal(pk2[name], pk1[name], err_msg=name)
    assert pk1["flags"][2] & lsp.FLAG_BAD_OFFSETS and pk1["flags"][7] & lsp.FLAG_BAD_OFFSETS
    assert not (pk1["flags"][0] & lsp.FLAG_BAD_OFFSETS)
    plan.close()


def test_host_group_count_rule(env, small_batch):
    """Clamp to n_obj / 2, one pass below 256 MiB by default, one-object plans
    in one pass, negative counts rejected."""
    lsp, torch, dev = env
    b, _ = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    assert plan.host_parts() == 1
    import ctypes
    v = ctypes.c_int32()
    assert lsp.lib().lsp_plan_get_host_parts(plan._h, 256 << 20, ctypes.byref(v)) == 0
    assert v.value == 8
    assert plan.host_parts(power=False) == 1  # inputs under 64 MiB: one pass
    plan.set_host_parts(100)
    assert plan.host_parts() == b.n_obj // 2
    assert plan.host_parts(power=False) == b.n_obj // 2
    with pytest.raises(lsp.LSPError):
        plan.set_host_parts(-1)
    plan.close()
    one = lsp.Plan(1, 500, g)
    one.set_host_parts(4)
    assert one.host_parts() == 1
    one.close()
    big = lsp.Plan(1000, 6_000_000, g)  # 72 MB of FP32 inputs: streamed in 4 groups
    assert big.host_parts(power=False) == 4
    big.close()


@pytest.mark.parametrize("parts", [2, 4, 7])
def test_peaks_only_host_call_streams_inputs_in_groups(env, parts):
    """The host entry point without a periodogram streams its inputs in object
    groups whose observation counts grow four-fold (each group's copy overlaps
    the previous group's kernels, Section 3.5): the peaks equal the device
    path's bit for bit, from pageable and page-locked inputs that start past
    offset 0.  The staging buffers hold other data before each grouped call,
    so a range that a group failed to copy would show."""
    lsp, torch, dev = env
    b = synth.ragged_lognormal(600, seed=31, grid=synth.Grid(0.24, 12.0, 3001))
    pad = 5
    t = np.concatenate([np.linspace(1.0, 2.0, pad), b.t])
    y = np.concatenate([np.ones(pad, np.float32), b.y.astype(np.float32)])
    off = b.offsets + pad
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    plan = lsp.Plan(b.n_obj, t.size, g, top_k=3)
    td = _dev(torch, dev, t, torch.float64)
    yd = _dev(torch, dev, y, torch.float32)
    od = _dev(torch, dev, off, torch.int64)
    pk_dev = plan.peaks_buffer(dev)
    plan.execute(td, yd, od, peaks=pk_dev)
    torch.cuda.synchronize()
    want = lsp.peaks_to_numpy(pk_dev)
    pinned = (torch.from_numpy(t).pin_memory(), torch.from_numpy(y).pin_memory(),
              torch.from_numpy(off).pin_memory())
    for inputs in ((t, y, off), pinned):
        plan.set_host_parts(1)
        plan.execute_host(t + 0.37, np.roll(y, 7), off)  # other data into the staging buffers
        plan.set_host_parts(parts)
        assert plan.host_parts(power=False) == parts
        got = plan.execute_host(*inputs)
        for name in lsp.PEAK_DTYPE.names:
            np.testing.assert_array_equal(got[name], want[name], err_msg=name)
    plan.close()


def test_fixed_point_sincos_matches_cuda(env):
    """The FP64 seeds' sin/cos (256-entry table of e^{2 pi i j/256} plus a
    Taylor series of the remaining angle) against CUDA's sincospi on 4e6
    phases, the table points and their neighbours included: within a few FP64
    ulp of 1."""
    lsp, torch, dev = env
    import ctypes
    err = ctypes.c_double(-1.0)
    assert lsp.lib().lsp_probe_sincos_fixed64(4_000_000, 12345, ctypes.byref(err), None) == 0
    assert 0.0 <= err.value <= 1e-15, err.value


def test_fma_rate_probe_is_plausible(env):
    # ceilings for the roofline fractions: below the nominal unit counts at the
    # highest SM clock of the part (2.07 GHz), and not far below them
    lsp, torch, dev = env
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    r = lsp.probe_fma_rates(dev)
    f32_nominal = n_sm * 128 * 2.07e9
    assert 0.5 * f32_nominal < r["f32"] <= 1.02 * f32_nominal, r
    assert 0.5 * f32_nominal < r["f32x2"] <= 1.02 * f32_nominal, r
    assert 0.3 * n_sm * 2 * 2.07e9 < r["f64"] <= 1.02 * n_sm * 2 * 2.07e9, r


# ------------------------------------------- ablations (Table 3, Table 6)
ABLATIONS = [(trig, staging) for staging in (0, 1) for trig in (0, 1, 2) if trig or staging]


@pytest.mark.parametrize("trig,staging", ABLATIONS, ids=lambda v: str(v))
def test_ablation_kernels_match_oracle(env, small_batch, trig, staging):
    # per-pair SFU / accurate sin-cos and global-memory observation reads:
    # the same periodogram within the FP32 tolerance
    lsp, torch, dev = env
    b, ref = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    plan.set_config(k_reseed=16, freqs_per_thread=16, block_threads=128, packed=0, obs_split=1,
                    trig=trig, staging=staging)
    assert plan.config["trig"] == trig and plan.config["staging"] == staging
    power = torch.empty((b.n_obj, g.n_f), dtype=torch.float32, device=dev)
    pk = lsp.peaks_to_numpy(plan.execute(t, y, off, power=power))
    err = np.max(np.abs(power.cpu().numpy().astype(np.float64) - ref["fp32"]["power"]))
    assert err <= TOL32, err
    for o in range(b.n_obj):
        assert_argmax_close(pk["idx"][o], ref["fp32"]["arg_idx"][o], ref["fp32"]["power"][o])
    plan.close()


def test_ablation_configs_are_checked(env, small_batch):
    lsp, torch, dev = env
    b, _ = small_batch
    plan = lsp.Plan(b.n_obj, b.t.size, lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f))
    for bad in (dict(trig=3), dict(staging=2), dict(trig=1, packed=1, freqs_per_thread=32),
                dict(trig=1, k_reseed=8, freqs_per_thread=8)):
        cfg = dict(k_reseed=16, freqs_per_thread=16, block_threads=128, packed=0, obs_split=1, trig=0, staging=0)
        cfg.update(bad)
        with pytest.raises(lsp.LSPError):
            plan.set_config(**cfg)
    plan.close()


def test_autotune_records_trials_including_ablations(env, small_batch, tmp_path):
    lsp, torch, dev = env
    b, ref = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    cfg, trials = plan.autotune(t, y, off, cache_path=str(tmp_path / "t.jsonl"), ablations=True,
                                return_trials=True)
    seen = {(tr["config"]["trig"], tr["config"]["staging"]) for tr in trials}
    assert set(ABLATIONS) <= seen
    for tr in trials:
        assert tr["passed"] and tr["ms"] > 0 and tr["max_err"] <= TOL32, tr
    assert min(tr["ms"] for tr in trials) == pytest.approx(
        min(tr["ms"] for tr in trials if tr["config"] == cfg), rel=1e-6)
    pk = lsp.peaks_to_numpy(plan.execute(t, y, off))
    for o in range(b.n_obj):
        assert_argmax_close(pk["idx"][o], ref["fp32"]["arg_idx"][o], ref["fp32"]["power"][o])
    plan.close()


def test_autotune_ex_rejects_bad_arguments(env, small_batch):
    import ctypes
    lsp, torch, dev = env
    b, _ = small_batch
    g = lsp.Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = _dev(torch, dev, b.t, torch.float64)
    y = _dev(torch, dev, b.y, torch.float32)
    off = _dev(torch, dev, b.offsets, torch.int64)
    plan = lsp.Plan(b.n_obj, b.t.size, g)
    P = ctypes.c_void_p
    n = ctypes.c_int32(-1)
    st = lsp.lib().lsp_plan_autotune_ex(plan._h, P(t.data_ptr()), P(y.data_ptr()), P(off.data_ptr()), None, 2,
                                        None, 0, ctypes.byref(n), None)
    assert st == 1 and n.value == 0  # LSP_E_ARG: unknown flag
    st = lsp.lib().lsp_plan_autotune_ex(plan._h, P(t.data_ptr()), P(y.data_ptr()), P(off.data_ptr()), None, 0,
                                        None, 4, None, None)
    assert st == 1  # trials NULL with max_trials > 0
    plan.close()

