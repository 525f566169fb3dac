"""GPU parity of the CUDA MrDFT against the FP64 oracle, through the C ABI.

Every input comes from the seeded generators in paper_1507_02525_gb300.inputs;
every expected value from oracle/.  Sizes run from N = 2 (the degenerate
level-1-only case) through the tile (2^12), window (2^13, 2^14) and two-pass
(2^15 ..) regimes to the full 2^24 signal and the 2^26 maximum.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1507_02525_gb300 import _lib, api, inputs  # noqa: E402

from tests._parity import ABS_FRAC, REL_PER_LEVEL, check_adjoint, check_forward_levels  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def run_forward(plan, x_np):
    """Forward through the C ABI with torch-allocated device buffers."""
    xt = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.status_poll()
    return y.cpu().numpy()


def run_adjoint(plan, gy_np):
    gyt = torch.from_numpy(np.ascontiguousarray(gy_np)).cuda()
    gx = torch.empty(plan.in_elems, dtype=torch.complex64, device="cuda")
    plan.adjoint(gyt.data_ptr(), gx.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.status_poll()
    return gx.cpu().numpy()


def split_out(y, lengths):
    out, o = [], 0
    for n in lengths:
        m = int(n).bit_length() - 1
        out.append(y[o:o + m * n].reshape(m, n))
        o += m * n
    return out


def split_in(x, lengths):
    out, o = [], 0
    for n in lengths:
        out.append(x[o:o + n])
        o += n
    return out


# ------------------------------------------------------------------ forward

@pytest.mark.parametrize("m", list(range(1, 21)))
def test_forward_single(oracle, m):
    N = 1 << m
    x = inputs.complex_signals(1, N, seed=1000 + m)[0]
    plan = _lib.Plan([N], 1)
    y = run_forward(plan, x).reshape(m, N)
    ref = oracle.forward(x.astype(np.complex128))
    check_forward_levels(y, ref, x, f"N=2^{m}")


@pytest.mark.parametrize("m", [5, 6, 7, 9, 11, 12])
@pytest.mark.parametrize("real", [False, True])
def test_forward_lone_signal_levels_parallel(oracle, m, real):
    """A plan of one signal of 2^5..2^12 samples computes every level in a CTA
    of its own (levels_parallel, the default); with the option off it runs
    the in-tile recursion. Both against the oracle, and the default path bit
    for bit the same on a second call and under graph replay."""
    N = 1 << m
    x = (inputs.real_signals(1, N, seed=70 + m) if real else inputs.complex_signals(1, N, seed=70 + m))[0]
    ref = oracle.forward(x.astype(np.complex128))
    ys = []
    for opts, graph in (({}, False), ({}, True), ({"levels_parallel": False}, False)):
        plan = _lib.Plan([N], 1, real_input=real, graph=graph, opts=opts)
        assert plan.opts()["levels_parallel"] is (opts.get("levels_parallel", True))
        y = run_forward(plan, x)
        np.testing.assert_array_equal(y, run_forward(plan, x))
        check_forward_levels(y.reshape(m, N), ref, x, f"lone N=2^{m} {opts}")
        ys.append(y)
    np.testing.assert_array_equal(ys[0], ys[1])


@pytest.mark.parametrize("m", [5, 6, 8, 10, 12])
def test_adjoint_lone_signal_levels_parallel(oracle, m):
    """The adjoint of a lone 2^5..2^12 signal: every level's share of x_bar in
    a CTA of its own, summed by the last CTA to finish -- against the oracle's
    adjoint, bit for bit the same on repeated calls and under graph replay, and
    against the in-tile path (levels_parallel off)."""
    N = 1 << m
    gy = inputs.targets(1, N, seed=90 + m)[0]  # [m, N]
    ref = oracle.adjoint(gy.astype(np.complex128))
    outs = []
    for opts, graph in (({}, False), ({}, True), ({"levels_parallel": False}, False)):
        plan = _lib.Plan([N], 1, graph=graph, opts=opts)
        gx = run_adjoint(plan, gy.reshape(-1))
        for _ in range(2):
            np.testing.assert_array_equal(gx, run_adjoint(plan, gy.reshape(-1)))
        check_adjoint(gx, ref, gy, f"lone N=2^{m} {opts}")
        outs.append(gx)
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("m", [5, 8, 12, 13, 15])
def test_forward_real_input(oracle, m):
    N = 1 << m
    x = inputs.real_signals(3, N, seed=50 + m)
    plan = _lib.Plan([N], 3, real_input=True)
    y = run_forward(plan, x.reshape(-1)).reshape(3, m, N)
    for s in range(3):
        ref = oracle.forward(x[s].astype(np.complex128))
        check_forward_levels(y[s], ref, x[s], f"real N=2^{m} s={s}")


@pytest.mark.parametrize("B,m", [(8, 10), (3, 16), (256, 6), (5, 5), (130, 7), (2, 14)])
def test_forward_uniform_batch(oracle, B, m):
    N = 1 << m
    x = inputs.complex_signals(B, N, seed=7 * B + m)
    plan = _lib.Plan([N], B)
    y = run_forward(plan, x.reshape(-1)).reshape(B, m, N)
    for s in range(B):
        ref = oracle.forward(x[s].astype(np.complex128))
        check_forward_levels(y[s], ref, x[s], f"B={B} N=2^{m} s={s}")


@pytest.mark.parametrize("real", [False, True])
def test_forward_ragged(oracle, real):
    rng = np.random.default_rng(77)
    ks = list(rng.integers(1, 18, size=40)) + [1, 2, 3, 4, 12, 13, 14, 15, 17]
    rng.shuffle(ks)
    lengths = [1 << int(k) for k in ks]
    total = sum(lengths)
    x = (inputs.real_signals(1, total, seed=78)[0] if real
         else inputs.complex_signals(1, total, seed=78)[0])
    plan = _lib.Plan(lengths, len(lengths), real_input=real)
    assert plan.out_elems == sum((n.bit_length() - 1) * n for n in lengths)
    ys = split_out(run_forward(plan, x), lengths)
    for s, (xs, ys_) in enumerate(zip(split_in(x, lengths), ys)):
        ref = oracle.forward(xs.astype(np.complex128))
        check_forward_levels(ys_, ref, xs, f"ragged s={s} N={len(xs)}")


@pytest.mark.parametrize("tree", [True, False])
@pytest.mark.parametrize("seg_log", [13, 15, 16, 23])
@pytest.mark.parametrize("dual", [True, False])
def test_forward_dual_cols_ragged(oracle, seg_log, dual, tree):
    """Two-pass levels paired in one cols pass (and not): signals that end at
    the lower level of a pair take the plain cols pass for their windows.
    The levels above the segment size run as a tree of per-window launches
    (tree) or level by level after every segment (not tree)."""
    lengths = [1 << k for k in (15, 16, 17, 15, 18, 16, 19)]
    total = sum(lengths)
    x = inputs.complex_signals(1, total, seed=88)[0]
    opts = {"dual_cols": dual, "fwd_tree": tree}
    plan = _lib.Plan(lengths, len(lengths), seg_log=seg_log, streams=2, opts=opts)
    assert plan.opts()["dual_cols"] == dual and plan.opts()["fwd_tree"] == tree
    # without tails a pair of levels saves one launch in each direction (a pair
    # with a tail takes cols2 + cols + rows + rows, as many as two levels)
    uni = _lib.Plan([1 << 18], 2, seg_log=seg_log, opts=opts).info()
    base = _lib.Plan([1 << 18], 2, seg_log=seg_log, opts=dict(opts, dual_cols=False)).info()
    if dual and seg_log >= 15:
        assert uni["adj_launches"] < base["adj_launches"]
        if not tree or seg_log >= 18:
            assert uni["fwd_launches"] < base["fwd_launches"]
    elif not dual:
        assert uni == base
    ys = split_out(run_forward(plan, x), lengths)
    for s, (xs, ys_) in enumerate(zip(split_in(x, lengths), ys)):
        ref = oracle.forward(xs.astype(np.complex128))
        check_forward_levels(ys_, ref, xs, f"dual={dual} S={seg_log} s={s} N={len(xs)}")


@pytest.mark.parametrize("pf", [True, False])
@pytest.mark.parametrize("cb", [9, 10, 11])
@pytest.mark.parametrize("m", [15, 16, 19, 22])
def test_forward_two_pass_split(oracle, cb, m, pf):
    """The splits of the two-pass levels, h = Q C with C = 2^max(i - 12, cb),
    with the rows CTAs that prefetch the children into shared memory (pf)
    and the ones that read them in the last FFT pass (not pf)."""
    N = 1 << m
    x = inputs.complex_signals(1, N, seed=300 + m)[0]
    y = run_forward(_lib.Plan([N], 1, opts={"fwd_cb": cb, "fwd_rows_prefetch": pf}), x).reshape(m, N)
    x128 = x.astype(np.complex128)
    xn = float(np.linalg.norm(x128))
    for i in range(13, m + 1):
        ref = oracle.forward_level(x128, i)
        d = y[i - 1].astype(np.complex128) - ref
        assert np.linalg.norm(d) / np.linalg.norm(ref) <= REL_PER_LEVEL * i, f"C=2^{cb} level {i}"
        assert np.abs(d).max() <= ABS_FRAC * xn, f"C=2^{cb} level {i} max abs"


def test_forward_graph_replay(oracle):
    N, B = 1 << 15, 2
    x = inputs.complex_signals(B, N, seed=5)
    plan = _lib.Plan([N], B, graph=True)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            plan.forward(xt.data_ptr(), y.data_ptr(), s.cuda_stream)
    s.synchronize()
    y1 = y.cpu().numpy().reshape(B, 15, N)
    plan2 = _lib.Plan([N], B)
    y2 = run_forward(plan2, x.reshape(-1)).reshape(B, 15, N)
    np.testing.assert_array_equal(y1, y2)  # graph replay = direct launch, bit for bit
    ref = oracle.forward(x[1].astype(np.complex128))
    check_forward_levels(y1[1], ref, x[1], "graph")


@pytest.mark.parametrize("seg_log,streams", [(14, 4), (16, 3), (20, 2), (21, 4)])
def test_forward_tree_long_signals(oracle, seg_log, streams):
    """Signals several segments long (the forward runs their upper levels as a
    tree of per-window launches across the worker streams), repeated under
    graph replay: every level of every signal against the oracle."""
    lengths = [1 << 20, 1 << 17, 1 << 22, 1 << 15]
    x = inputs.complex_signals(1, sum(lengths), seed=123)[0]
    plan = _lib.Plan(lengths, len(lengths), graph=True, seg_log=seg_log, streams=streams)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        y.fill_(float("nan"))
        plan.forward(xt.data_ptr(), y.data_ptr(), sp)
    torch.cuda.synchronize()
    plan.status_poll()
    ys = split_out(y.cpu().numpy(), lengths)
    for s, (xs, ys_) in enumerate(zip(split_in(x, lengths), ys)):
        check_forward_levels(ys_, oracle.forward(xs.astype(np.complex128)), xs, f"S={seg_log} s={s}")


def test_forward_deterministic():
    N = 1 << 17
    x = inputs.complex_signals(1, N, seed=9)[0]
    plan = _lib.Plan([N], 1)
    np.testing.assert_array_equal(run_forward(plan, x), run_forward(plan, x))


def test_forward_host_entry(oracle):
    N, B = 1 << 13, 3
    x = inputs.complex_signals(B, N, seed=21)
    plan = _lib.Plan([N], B)
    y_host = np.empty(plan.out_elems, dtype=np.complex64)
    plan.forward_host(x.ctypes.data, y_host.ctypes.data, 0)
    np.testing.assert_array_equal(y_host, run_forward(plan, x.reshape(-1)))


@pytest.mark.parametrize("case", ["phases", "tile_split", "bitrev", "many_runs", "lone"])
def test_forward_host_overlapped_copies(oracle, case):
    """mrdft_forward_host copies each finished part of the output (the in-tile
    levels after the tile launch, the segment levels after the segments, the
    rest at the end) while the forward goes on; every case must equal the
    device-buffer forward bit for bit, into pinned and pageable host memory,
    over repeated calls."""
    if case == "many_runs":
        lengths = [1 << int(m) for m in np.random.default_rng(5).integers(3, 15, size=100)]
    elif case == "lone":  # one small signal: one CTA per level, copied after that launch
        lengths = [1 << 12]
    else:
        lengths = [1 << 20, 1 << 17, 1 << 13, 1 << 5, 1 << 3]
    opts = {"tile_split": 2} if case == "tile_split" else {}
    plan = _lib.Plan(lengths, len(lengths), graph=True, seg_log=16, streams=3, opts=opts, bitrev=case == "bitrev")
    x = inputs.complex_signals(1, sum(lengths), seed=31)[0]
    want = run_forward(plan, x)
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.empty(plan.out_elems, dtype=torch.complex64).pin_memory()
    for _ in range(2):
        yp.fill_(float("nan"))
        plan.forward_host(xp.data_ptr(), yp.data_ptr(), torch.cuda.current_stream().cuda_stream)
        np.testing.assert_array_equal(yp.numpy(), want)
    y_pageable = np.full(plan.out_elems, np.nan, dtype=np.complex64)
    plan.forward_host(x.ctypes.data, y_pageable.ctypes.data, 0)
    np.testing.assert_array_equal(y_pageable, want)
    plan.status_poll()


def test_forward_api_shapes(oracle):
    x = inputs.complex_signals(2, 256, seed=3)
    y = api.mrdft(torch.from_numpy(x).cuda())
    assert y.shape == (2, 8, 256) and y.dtype == torch.complex64
    y1 = api.mrdft(torch.from_numpy(x[0]).cuda())
    assert y1.shape == (8, 256)
    # a lone signal takes the one-CTA-per-level path, the batch the in-tile
    # recursion: the same transform, rounded differently
    ref = oracle.forward(x[0].astype(np.complex128))
    check_forward_levels(y1.cpu().numpy(), ref, x[0], "lone")
    check_forward_levels(y[0].cpu().numpy(), ref, x[0], "batch")


def test_closed_forms_on_gpu():
    """Impulse at a window start -> all-ones spectra; constant -> DC only."""
    N, m = 1 << 14, 14
    x = np.zeros(N, np.complex64)
    x[0] = 1.0
    y = run_forward(_lib.Plan([N], 1), x).reshape(m, N)
    for i in range(1, m + 1):
        L = 1 << i
        np.testing.assert_allclose(y[i - 1][:L], 1.0, atol=1e-6)
        np.testing.assert_allclose(y[i - 1][L:], 0.0, atol=1e-6)
    c = np.full(N, 0.5 - 0.25j, np.complex64)
    y = run_forward(_lib.Plan([N], 1), c).reshape(m, N)
    for i in range(1, m + 1):
        L = 1 << i
        blk = y[i - 1].reshape(-1, L)
        np.testing.assert_allclose(blk[:, 0], (0.5 - 0.25j) * L, rtol=1e-6)
        assert np.abs(blk[:, 1:]).max() <= 1e-6 * L


# -------------------------------------------------------- full-size workloads

@pytest.fixture(scope="module")
def big_signal():
    x = inputs.complex_signals(1, 1 << 24, seed=1)[0]
    plan = _lib.Plan([1 << 24], 1)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.status_poll()
    return x, y.view(24, 1 << 24)


def test_single_16m_every_level(oracle, big_signal):
    """N = 2^24: every level compared in full with the oracle's FFT path.

    The relative error of every level must also stay within a tenth of the
    2e-6 i budget: the twiddles of the large levels are products of at most
    three FP64-rounded-once table values (about 3 ulp each), and this bounds
    what those extra roundings cost."""
    x, y = big_signal
    x128 = x.astype(np.complex128)
    xn = float(np.linalg.norm(x128))
    fracs = []
    for i in range(1, 25):
        ref = oracle.forward_level(x128, i)
        d = y[i - 1].cpu().numpy().astype(np.complex128) - ref
        rel = np.linalg.norm(d) / np.linalg.norm(ref)
        fracs.append(rel / (2e-6 * i))
        assert rel <= 2e-6 * i, f"level {i}: rel {rel:.3e}"
        assert np.abs(d).max() <= 1e-5 * xn, f"level {i}: max abs"
    print("fraction of the per-level budget used, levels 1..24:", " ".join(f"{f:.4f}" for f in fracs))
    assert max(fracs) <= 0.1, fracs


def _level_error_gpu(y_level, ref_gpu, xn):
    d = y_level.to(torch.complex128) - ref_gpu
    rel = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(ref_gpu))
    return rel, float(d.abs().max()) / xn


def test_single_16m_every_exec_shape(oracle):
    """N = 2^24 planned with every execution shape the autotuner can pick
    (segment size x worker streams, including the shapes bench.py timed) and
    the library default: every level of every plan compared element by
    element with the oracle (the comparison runs on the GPU in FP64)."""
    from paper_1507_02525_gb300 import autotune
    N = 1 << 24
    x = inputs.complex_signals(1, N, seed=1)[0]
    xt = torch.from_numpy(x).cuda()
    sp = torch.cuda.current_stream().cuda_stream
    shapes = [(0, 0)] + list(autotune.DEFAULT_CANDIDATES)
    ys = {}
    for seg, st in shapes:
        plan = _lib.Plan([N], 1, graph=True, seg_log=seg or None, streams=st or None)
        y = torch.empty((24, N), dtype=torch.complex64, device="cuda")
        for _ in range(2):  # capture, then replay
            plan.forward(xt.data_ptr(), y.data_ptr(), sp)
        torch.cuda.synchronize()
        plan.status_poll()
        plan.close()
        ys[(seg, st)] = y
    x128 = x.astype(np.complex128)
    xn = float(np.linalg.norm(x128))
    for i in range(1, 25):
        ref = torch.from_numpy(oracle.forward_level(x128, i)).cuda()
        for shape, y in ys.items():
            rel, mx = _level_error_gpu(y[i - 1], ref, xn)
            assert rel <= 2e-6 * i, f"shape {shape} level {i}: rel {rel:.3e}"
            assert mx <= 1e-5, f"shape {shape} level {i}: max abs / ||x|| {mx:.3e}"
        del ref
    del ys, xt
    torch.cuda.empty_cache()


def test_adjoint_16m_elementwise(oracle):
    """N = 2^24 adjoint, element by element against the oracle's FFT adjoint,
    for the default execution shape and the shapes the autotuner picks from."""
    N = 1 << 24
    g = inputs.targets(1, N, seed=24)[0]
    ref = torch.from_numpy(oracle.adjoint(g.astype(np.complex128), "fft")).cuda()
    gt = torch.from_numpy(g.reshape(-1)).cuda()
    gn = float(torch.linalg.vector_norm(gt.to(torch.complex128)))
    sp = torch.cuda.current_stream().cuda_stream
    for seg, st in [(0, 0), (23, 2), (21, 4), (20, 4), (26, 1)]:
        plan = _lib.Plan([N], 1, graph=True, seg_log=seg or None, streams=st or None)
        gx = torch.empty(N, dtype=torch.complex64, device="cuda")
        for _ in range(2):
            plan.adjoint(gt.data_ptr(), gx.data_ptr(), sp)
        torch.cuda.synchronize()
        plan.status_poll()
        plan.close()
        d = gx.to(torch.complex128) - ref
        rel = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(ref))
        mx = float(d.abs().max())
        assert rel <= 1e-5, f"shape {(seg, st)}: adjoint rel {rel:.3e}"
        assert mx <= 1e-5 * gn, f"shape {(seg, st)}: adjoint max abs {mx:.3e}"
    del ref, gt
    torch.cuda.empty_cache()


@pytest.mark.parametrize("rows14", [True, False])
def test_single_16m_top_rows_variant(oracle, big_signal, rows14):
    """Levels 23-24 with the rows CTAs that read the children in the last FFT
    pass: level 24 (C = 2^12) in CTAs of 2^14 points (rows14) or 2^13."""
    x, _ = big_signal
    plan = _lib.Plan([1 << 24], 1, opts={"fwd_rows_prefetch": False, "fwd_rows14": rows14})
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.status_poll()
    x128 = x.astype(np.complex128)
    xn = float(np.linalg.norm(x128))
    for i in (23, 24):
        ref = oracle.forward_level(x128, i)
        d = y.view(24, 1 << 24)[i - 1].cpu().numpy().astype(np.complex128) - ref
        assert np.linalg.norm(d) / np.linalg.norm(ref) <= 2e-6 * i, f"level {i}"
        assert np.abs(d).max() <= 1e-5 * xn, f"level {i} max abs"
    del y, xt
    torch.cuda.empty_cache()


def test_single_16m_sampled_bins(oracle, big_signal):
    """Independent check: bins evaluated one by one with the direct sum of Eq. 1."""
    x, y = big_signal
    x128 = x.astype(np.complex128)
    xn = float(np.linalg.norm(x128))
    rng = np.random.default_rng(123)
    for i in (1, 2, 7, 12, 13, 15, 18, 20, 24):
        for pos in list(rng.integers(0, 1 << 24, size=3)) + [0, (1 << 24) - 1]:
            ref = oracle.bin_value(x128, i, int(pos))
            got = complex(y[i - 1, int(pos)].item())
            assert abs(got - ref) <= 1e-5 * xn, f"level {i} pos {pos}"


def test_batch_256x64k(oracle):
    """The 256 x 2^16 workload: every level of every signal against the oracle."""
    B, N, m = 256, 1 << 16, 16
    x = inputs.complex_signals(B, N, seed=2)
    y = run_forward(_lib.Plan([N], B), x.reshape(-1)).reshape(B, m, N)
    for s in range(B):
        ref = oracle.forward(x[s].astype(np.complex128))
        check_forward_levels(y[s], ref, x[s], f"batch s={s}")


def test_ragged_1024_graph_replay(oracle):
    """The ragged workload (1024 real signals, N = 2^k, k ~ U{8..18}) planned
    for graph replay and replayed three times: every replay bit-identical to a
    direct launch, every level of every signal against the oracle."""
    lengths, samples = inputs.ragged_real()
    lengths = [int(v) for v in lengths]
    plan = _lib.Plan(lengths, len(lengths), real_input=True, graph=True)
    xt = torch.from_numpy(samples).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    outs = []
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(s):
            y.fill_(float("nan"))  # on the replay stream: ordered before the graph
            plan.forward(xt.data_ptr(), y.data_ptr(), s.cuda_stream)
        s.synchronize()
        outs.append(y.cpu().numpy())
    plan.status_poll()
    assert plan.graph_stats()["captures"] == 1
    direct = run_forward(_lib.Plan(lengths, len(lengths), real_input=True), samples)
    for o in outs:
        np.testing.assert_array_equal(o, direct)
    ys = split_out(outs[-1], lengths)
    xs = split_in(samples, lengths)
    for k in range(len(lengths)):
        ref = oracle.forward(xs[k].astype(np.complex128))
        check_forward_levels(ys[k], ref, xs[k], f"ragged1024 s={k}")


def test_maximum_length_2_26(oracle):
    """The largest length a plan accepts, checked on sampled bins."""
    N = 1 << 26
    x = inputs.complex_signals(1, N, seed=26)[0]
    plan = _lib.Plan([N], 1)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    plan.status_poll()
    y = y.view(26, N)
    x128 = x.astype(np.complex128)
    xn = float(np.linalg.norm(x128))
    for i, pos in [(1, 5), (5, N - 1), (12, 123456), (16, 7_000_001), (21, 3), (23, 40_000_001),
                   (24, N - 3), (25, 12_345_679), (25, (1 << 25) + 7), (26, 0), (26, N // 2 + 1)]:
        ref = oracle.bin_value(x128, i, pos)
        assert abs(complex(y[i - 1, pos].item()) - ref) <= 1e-5 * xn, f"level {i} pos {pos}"
    del y, xt
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("m", list(range(1, 19)))
def test_adjoint_single(oracle, m):
    N = 1 << m
    g = inputs.targets(1, N, seed=300 + m)[0]
    gx = run_adjoint(_lib.Plan([N], 1), g.reshape(-1))
    ref = oracle.adjoint(g.astype(np.complex128))
    check_adjoint(gx, ref, g, f"N=2^{m}")


def test_adjoint_ragged(oracle):
    rng = np.random.default_rng(88)
    ks = list(rng.integers(1, 17, size=30)) + [1, 4, 5, 12, 13, 14, 15, 16]
    rng.shuffle(ks)
    lengths = [1 << int(k) for k in ks]
    plan = _lib.Plan(lengths, len(lengths))
    gy = inputs.complex_signals(1, plan.out_elems, seed=89)[0]
    gx = split_in(run_adjoint(plan, gy), lengths)
    gys = split_out(gy, lengths)
    for s in range(len(lengths)):
        ref = oracle.adjoint(gys[s].astype(np.complex128))
        check_adjoint(gx[s], ref, gys[s], f"ragged s={s}")


@pytest.mark.parametrize("seg_log", [15, 16, 23])
@pytest.mark.parametrize("dual", [True, False])
def test_adjoint_dual_cols_ragged(oracle, seg_log, dual):
    """Adjoint with two-pass levels paired in one cols pass (and not),
    including signals that end at the lower level of a pair."""
    lengths = [1 << k for k in (15, 16, 17, 15, 18, 16, 19, 20)]
    plan = _lib.Plan(lengths, len(lengths), seg_log=seg_log, streams=2, opts={"dual_cols": dual})
    gy = inputs.complex_signals(1, plan.out_elems, seed=90)[0]
    gx = split_in(run_adjoint(plan, gy), lengths)
    gys = split_out(gy, lengths)
    for s in range(len(lengths)):
        ref = oracle.adjoint(gys[s].astype(np.complex128))
        check_adjoint(gx[s], ref, gys[s], f"dual={dual} S={seg_log} s={s}")


def test_adjoint_short_signals_first(oracle):
    """Signals that end inside a tile ahead of longer ones: the accumulator of
    the large levels holds only the longer signals and is indexed by their own
    offsets, not by their position in x."""
    lengths = [1 << 12] * 64 + [1 << 8] * 64 + [1 << 17] + [1 << 10] * 8 + [1 << 15]
    plan = _lib.Plan(lengths, len(lengths))
    gy = inputs.complex_signals(1, plan.out_elems, seed=93)[0]
    gx = split_in(run_adjoint(plan, gy), lengths)
    gys = split_out(gy, lengths)
    for s in (0, 63, 64, 127, 128, 129, 136):
        ref = oracle.adjoint(gys[s].astype(np.complex128))
        check_adjoint(gx[s], ref, gys[s], f"short-first s={s} N={lengths[s]}")


def test_adjoint_dot_product():
    """<M x, g> = <x, M^H g> with both sides on the GPU (N = 2^18, batch 4)."""
    B, N = 4, 1 << 18
    x = inputs.complex_signals(B, N, seed=11)
    g = inputs.targets(B, N, seed=12)
    plan = _lib.Plan([N], B)
    y = run_forward(plan, x.reshape(-1)).astype(np.complex128)
    gx = run_adjoint(plan, g.reshape(-1)).astype(np.complex128)
    lhs = np.vdot(g.reshape(-1).astype(np.complex128), y)
    rhs = np.vdot(gx, x.reshape(-1).astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("seg_log", [12, 13, 14, 16])
def test_adjoint_long_signal_segments(oracle, seg_log):
    """Signals longer than a segment: the segments of one parent window run
    concurrently on worker streams and read the top level's propagation while
    transforming their own levels (repeated to give a race a chance)."""
    lengths = [1 << 18, 1 << 16, 1 << 17]
    plan = _lib.Plan(lengths, len(lengths), seg_log=seg_log, streams=4)
    gy = inputs.complex_signals(1, plan.out_elems, seed=91)[0]
    gys = split_out(gy, lengths)
    refs = [oracle.adjoint(g.astype(np.complex128)) for g in gys]
    for rep in range(3):
        gx = split_in(run_adjoint(plan, gy), lengths)
        for s in range(len(lengths)):
            check_adjoint(gx[s], refs[s], gys[s], f"S={seg_log} rep={rep} s={s}")


@pytest.mark.parametrize("cb,rows13", [(10, False), (10, True), (9, True)])
@pytest.mark.parametrize("m", [15, 18, 20])
def test_adjoint_rows_split(oracle, cb, rows13, m):
    """Adjoint splits h = Q C with C = 2^max(i - 12, cb): rows CTAs of 2^12
    points (4 residues) or 2^13 (8 residues) for C = 2^10, 2^13 for C = 2^9."""
    N = 1 << m
    plan = _lib.Plan([N], 2, opts={"adj_cb": cb, "adj_rows13": rows13})
    gy = inputs.complex_signals(1, plan.out_elems, seed=400 + m)[0]
    gx = run_adjoint(plan, gy)
    for s in range(2):
        g = gy[s * m * N:(s + 1) * m * N].reshape(m, N)
        check_adjoint(gx[s * N:(s + 1) * N], oracle.adjoint(g.astype(np.complex128)), g, f"C=2^{cb} rows13={rows13} m={m} s={s}")


def test_adjoint_dot_product_16m():
    """<M x, g> = <x, M^H g> at N = 2^24 with the default execution shape
    (two segments of 2^23 under one top level), sums in FP64 on the GPU."""
    N = 1 << 24
    plan = _lib.Plan([N], 1)
    gen = torch.Generator(device="cuda").manual_seed(24)
    x = torch.randn(N, dtype=torch.complex64, device="cuda", generator=gen)
    g = torch.randn(plan.out_elems, dtype=torch.complex64, device="cuda", generator=gen)
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    gx = torch.empty(N, dtype=torch.complex64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        plan.forward(x.data_ptr(), y.data_ptr(), sp)
        plan.adjoint(g.data_ptr(), gx.data_ptr(), sp)
        torch.cuda.synchronize()
        plan.status_poll()
        lhs = sum(torch.vdot(g[o:o + N].to(torch.complex128), y[o:o + N].to(torch.complex128)).item()
                  for o in range(0, plan.out_elems, N))
        rhs = torch.vdot(gx.to(torch.complex128), x.to(torch.complex128)).item()
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
    del x, g, y, gx
    torch.cuda.empty_cache()


def test_adjoint_dot_product_64m():
    """<M x, g> = <x, M^H g> at the maximum length N = 2^26 (top levels 24-26,
    C = 2^12..2^14), sums in FP64 on the GPU."""
    N = 1 << 26
    plan = _lib.Plan([N], 1)
    gen = torch.Generator(device="cuda").manual_seed(26)
    x = torch.randn(N, dtype=torch.complex64, device="cuda", generator=gen)
    g = torch.randn(plan.out_elems, dtype=torch.complex64, device="cuda", generator=gen)
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    gx = torch.empty(N, dtype=torch.complex64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    plan.forward(x.data_ptr(), y.data_ptr(), sp)
    plan.adjoint(g.data_ptr(), gx.data_ptr(), sp)
    torch.cuda.synchronize()
    plan.status_poll()
    lhs = sum(torch.vdot(g[o:o + N].to(torch.complex128), y[o:o + N].to(torch.complex128)).item()
              for o in range(0, plan.out_elems, N))
    rhs = torch.vdot(gx.to(torch.complex128), x.to(torch.complex128)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
    # the top level alone: the adjoint of level 26 is an unnormalised inverse DFT of the whole signal
    g.zero_()
    g[25 * N:26 * N] = torch.randn(N, dtype=torch.complex64, device="cuda", generator=gen)
    plan.adjoint(g.data_ptr(), gx.data_ptr(), sp)
    torch.cuda.synchronize()
    ref = torch.fft.ifft(g[25 * N:26 * N].to(torch.complex128)) * N
    err = (torch.linalg.vector_norm(gx.to(torch.complex128) - ref) / torch.linalg.vector_norm(ref)).item()
    assert err <= 1e-5, err
    del x, g, y, gx, ref
    torch.cuda.empty_cache()


def test_adjoint_grad_workload(oracle):
    """64 x 2^18 loss sum_i 2^-i ||Y_i - T_i||^2: gradient through autograd
    against the oracle's adjoint of the oracle's residual (sampled signals)."""
    B, N, m = 64, 1 << 18, 18
    x = inputs.complex_signals(B, N, seed=4)
    T = inputs.targets(B, N, seed=5)
    w = torch.tensor([2.0 ** -(i + 1) for i in range(m)], device="cuda").view(1, m, 1)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    Tt = torch.from_numpy(T).cuda()
    Y = api.MrDFT.apply(xt)
    loss = (w * (Y - Tt).abs() ** 2).sum()
    loss.backward()
    g = xt.grad.cpu().numpy()
    wn = 2.0 ** -np.arange(1, m + 1)
    for s in (0, 31, 63):
        Yr = oracle.forward(x[s].astype(np.complex128))
        gy = 2 * wn[:, None] * (Yr - T[s].astype(np.complex128))
        ref = oracle.adjoint(gy)
        rel = np.linalg.norm(g[s] - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, f"signal {s}: grad rel {rel:.3e}"


def test_autograd_finite_differences(oracle):
    """N = 2^8 slice: autograd gradient vs central differences of the FP64 oracle loss."""
    N, m = 256, 8
    x = inputs.complex_signals(1, N, seed=40)[0]
    T = inputs.targets(1, N, seed=41)[0].astype(np.complex128)
    wn = 2.0 ** -np.arange(1, m + 1)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    Y = api.MrDFT.apply(xt)
    loss = (torch.from_numpy(wn).cuda().float().view(m, 1)
            * (Y - torch.from_numpy(T.astype(np.complex64)).cuda()).abs() ** 2).sum()
    loss.backward()
    g = xt.grad.cpu().numpy().astype(np.complex128)
    x128 = x.astype(np.complex128)

    def L(v):
        return float((wn[:, None] * np.abs(oracle.forward(v) - T) ** 2).sum())

    eps = 1e-6
    rng = np.random.default_rng(0)
    for p in rng.choice(N, size=24, replace=False):
        for unit in (1.0, 1j):
            e = np.zeros(N, complex)
            e[p] = unit * eps
            fd = (L(x128 + e) - L(x128 - e)) / (2 * eps)
            an = g[p].real if unit == 1.0 else g[p].imag
            assert abs(fd - an) <= 1e-4 * max(1.0, abs(fd)), f"p={p} unit={unit}: fd {fd} vs {an}"


def test_autograd_real_input(oracle):
    N, m = 1 << 12, 12
    x = inputs.real_signals(2, N, seed=70)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    Y = api.MrDFT.apply(xt)
    (Y.abs() ** 2).sum().backward()
    g = xt.grad.cpu().numpy()
    for s in range(2):
        Yr = oracle.forward(x[s].astype(np.complex128))
        ref = oracle.adjoint(2 * Yr).real
        np.testing.assert_allclose(g[s], ref, rtol=0, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("B,m", [(1, 16), (4, 13)])
def test_matches_per_level_cufft(B, m):
    """Every level equals the batched FFT of its windows (cuFFT through torch.fft),
    within the same FP32 tolerance: an independent cross-check of the layout."""
    n = 1 << m
    x = torch.from_numpy(inputs.complex_signals(B, n, seed=77 + m)).cuda()
    y = api.mrdft(x)
    torch.cuda.synchronize()
    xn = float(torch.linalg.vector_norm(x.cpu().to(torch.complex128)))
    for i in range(1, m + 1):
        ref = torch.fft.fft(x.view(B, n >> i, 1 << i)).reshape(B, n).cpu().to(torch.complex128)
        got = y[:, i - 1, :].cpu().to(torch.complex128)
        rel = float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref))
        assert rel <= 2 * REL_PER_LEVEL * i, (i, rel)
        assert float((got - ref).abs().max()) <= 2 * ABS_FRAC * xn


@pytest.mark.parametrize("B,m,real", [(8, 3, False), (4, 12, False), (2, 17, False), (4, 15, True)])
def test_fused_loss_grad(oracle, B, m, real):
    """mrdft_loss_grad: Y, L = sum_i 2^-i ||Y_i - T_i||^2 and gx = adjoint of
    2^(1-i) (Y_i - T_i) in one call, against the oracle (FP64 forward, residual,
    adjoint) and against the unfused adjoint of the same residual."""
    N = 1 << m
    x = inputs.real_signals(B, N, seed=40 + m) if real else inputs.complex_signals(B, N, seed=40 + m)
    T = inputs.targets(B, N, seed=50 + m)
    xt = torch.from_numpy(x).cuda()
    Tt = torch.from_numpy(T).cuda()
    loss, y, g = api.mrdft_loss_grad(xt, Tt)
    torch.cuda.synchronize()
    wn = 2.0 ** -np.arange(1, m + 1)
    ys = y.cpu().numpy()
    gs = g.cpu().numpy()
    L_ref = 0.0
    for s in range(B):
        xs = x[s].astype(np.complex128)
        Yr = oracle.forward(xs)
        check_forward_levels(ys[s], Yr, xs, f"signal {s}")
        res = Yr - T[s].astype(np.complex128)
        L_ref += float((wn[:, None] * np.abs(res) ** 2).sum())
        gref = oracle.adjoint(2 * wn[:, None] * res)
        if real:
            gref = gref.real
        rel = np.linalg.norm(gs[s] - gref) / np.linalg.norm(gref)
        assert rel <= ADJ_REL_FUSED, f"signal {s}: gradient rel {rel:.3e}"
    assert abs(float(loss) - L_ref) <= 1e-5 * L_ref, (float(loss), L_ref)
    # unfused: the residual materialised, then the plain adjoint
    w = torch.tensor(wn, dtype=torch.float32, device="cuda").view(1, m, 1)
    gy = (2 * w * (y - Tt)).to(torch.complex64)
    g2 = api.mrdft_adjoint(gy)
    if real:
        g2 = g2.real
    d = (g2 - g).abs().max().item()
    assert d <= 1e-5 * g2.abs().max().item()


ADJ_REL_FUSED = 1e-5


def test_fused_loss_grad_graph_and_repeat():
    """The fused call under graph replay returns the same loss and gradient
    every time (the loss accumulator is reset on every call)."""
    B, m = 4, 16
    N = 1 << m
    xt = torch.from_numpy(inputs.complex_signals(B, N, seed=61)).cuda()
    Tt = torch.from_numpy(inputs.targets(B, N, seed=62)).cuda()
    l0, y0, g0 = api.mrdft_loss_grad(xt, Tt, graph=True)
    for _ in range(3):
        l1, y1, g1 = api.mrdft_loss_grad(xt, Tt, graph=True)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1) and torch.equal(g0, g1)
        assert abs(float(l1) - float(l0)) <= 1e-9 * abs(float(l0))


def test_autotuned_plan(oracle, tmp_path, monkeypatch):
    """The autotuner picks one of its candidates on the GPU, caches it, and a
    plan with the tuned shape still matches the oracle."""
    from paper_1507_02525_gb300 import autotune
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    cands = [(13, 1), (14, 2), (16, 4)]
    best = autotune.tune([1 << 16] * 8, 8, candidates=cands, reps=2)
    assert best in cands
    assert autotune.tune([1 << 16] * 8, 8, candidates=cands) == best  # cached
    x = inputs.complex_signals(8, 1 << 16, seed=71)
    plan = _lib.Plan([1 << 16], 8, seg_log=best[0], streams=best[1])
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    yn = y.cpu().numpy().reshape(8, 16, 1 << 16)
    for s in (0, 7):
        check_forward_levels(yn[s], oracle.forward(x[s].astype(np.complex128)), x[s], f"signal {s}")
    plan.close()


# ------------------------------------------------- bit-reversed output layout

def _bitrev_perm(i):
    k = np.arange(1 << i)
    r = np.zeros_like(k)
    for b in range(i):
        r |= ((k >> b) & 1) << (i - 1 - b)
    return r


def test_bitrev_permutation_is_the_papers_T():
    """The permutation the bit-reversed layout applies to a window of level i is
    the matrix T_{2^i} of Sec. 3 (built from its definition in oracle.matrices,
    itself pinned by the printed T_4 and T_8)."""
    from oracle import matrices
    for i in range(1, 7):
        v = np.arange(1 << i) + 1j * np.arange(1 << i)[::-1]
        np.testing.assert_array_equal(matrices.T(i) @ v, v[_bitrev_perm(i)])


@pytest.mark.parametrize("lengths", [[1 << 10], [1 << 16] * 3, [1 << 24],
                                     [1 << k for k in (3, 9, 13, 15, 12, 17, 4, 14, 20, 1)]])
def test_forward_bitrev_layout(oracle, lengths):
    """MRDFT_FLAG_BITREV: every window of every level holds the oracle's bins in
    the bit-reversed order T_{2^i} of Sec. 3 (tiny, in-tile, window and
    two-pass levels, a 2^24 signal, ragged lengths), and the same plan with
    graph replay gives the same bits; the adjoint is refused."""
    x = inputs.complex_signals(1, sum(lengths), seed=202)[0]
    plan = _lib.Plan(lengths, len(lengths), bitrev=True)
    y = run_forward(plan, x)
    gplan = _lib.Plan(lengths, len(lengths), bitrev=True, graph=True)
    xt = torch.from_numpy(x).cuda()
    yg = torch.empty(gplan.out_elems, dtype=torch.complex64, device="cuda")
    for _ in range(2):
        gplan.forward(xt.data_ptr(), yg.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yg.cpu().numpy(), y)
    ys = split_out(y, lengths)
    for s, (xs, ys_) in enumerate(zip(split_in(x, lengths), ys)):
        m = ys_.shape[0]
        x128 = xs.astype(np.complex128)
        ref = oracle.forward(x128) if m <= 20 else None
        for i in range(1, m + 1):
            nat = ref[i - 1] if ref is not None else oracle.forward_level(x128, i)
            want = nat.reshape(-1, 1 << i)[:, _bitrev_perm(i)].reshape(-1)
            d = ys_[i - 1].astype(np.complex128) - want
            assert np.linalg.norm(d) <= 2e-6 * i * np.linalg.norm(want), f"s={s} level {i}"
    with pytest.raises(_lib.MrdftError) as e:
        plan.adjoint(xt.data_ptr(), xt.data_ptr(), 0)
    assert e.value.status == _lib.MRDFT_EUNSUPPORTED


@pytest.mark.parametrize("seg_log", [12, 14, 17, 23])
def test_tile_first_both_directions(oracle, seg_log):
    """tile_first: the in-tile levels of every segment as one launch, ahead of
    the segments in the forward and after them in the adjoint (which then reads
    every segment's accumulator and level-13 propagation at the end)."""
    lengths = [1 << 18, 1 << 12, 1 << 16, 1 << 9, 1 << 15, 1 << 13]
    x = inputs.complex_signals(1, sum(lengths), seed=404)[0]
    plan = _lib.Plan(lengths, len(lengths), seg_log=seg_log, streams=3, opts={"tile_first": True})
    assert plan.opts()["tile_first"] is True
    ys = split_out(run_forward(plan, x), lengths)
    gy = inputs.complex_signals(1, plan.out_elems, seed=405)[0]
    gx = split_in(run_adjoint(plan, gy), lengths)
    gys = split_out(gy, lengths)
    for s, xs in enumerate(split_in(x, lengths)):
        check_forward_levels(ys[s], oracle.forward(xs.astype(np.complex128)), xs, f"S={seg_log} s={s}")
        check_adjoint(gx[s], oracle.adjoint(gys[s].astype(np.complex128)), gys[s], f"S={seg_log} s={s}")


@pytest.mark.parametrize("real", [False, True])
def test_tile_lean_forward(oracle, real):
    """tile_lean: the forward tile CTAs that fit three to an SM (work area
    sharing the level buffer, twiddles through L1): every length from 2^5 to
    2^16, packed tiles of short signals, ragged, real and complex input."""
    rng = np.random.default_rng(505)
    ks = list(range(5, 17)) + list(rng.integers(5, 13, size=40)) + [12] * 5 + [6] * 70
    rng.shuffle(ks)
    lengths = [1 << int(k) for k in ks]
    total = sum(lengths)
    x = (inputs.real_signals(1, total, seed=506)[0] if real
         else inputs.complex_signals(1, total, seed=506)[0])
    plan = _lib.Plan(lengths, len(lengths), real_input=real, opts={"tile_lean": True})
    assert plan.opts()["tile_lean"] is True
    ys = split_out(run_forward(plan, x), lengths)
    for s, xs in enumerate(split_in(x, lengths)):
        check_forward_levels(ys[s], oracle.forward(xs.astype(np.complex128)), xs, f"lean s={s} N={len(xs)}")


@pytest.mark.parametrize("m", [15, 16, 19, 21])
def test_forward_rows12(oracle, m):
    """fwd_rows12: the C = 2^9 two-pass levels in rows CTAs of 2^12 points."""
    N = 1 << m
    x = inputs.complex_signals(2, N, seed=600 + m)
    y = run_forward(_lib.Plan([N], 2, seg_log=20, opts={"fwd_rows12": True}), x.reshape(-1)).reshape(2, m, N)
    for s in range(2):
        check_forward_levels(y[s], oracle.forward(x[s].astype(np.complex128)), x[s], f"rows12 m={m} s={s}")


@pytest.mark.parametrize("split,seg_log,streams", [(2, 14, 3), (3, 15, 2), (4, 16, 4), (8, 13, 1)])
def test_tile_split_both_directions(oracle, split, seg_log, streams):
    """tile_split: the in-tile levels as several launches over groups of
    segments -- each forward segment waits only for its own group's tiles, each
    adjoint tile group only for its own segments -- repeated under graph replay."""
    lengths = [1 << 18, 1 << 12, 1 << 16, 1 << 9, 1 << 15, 1 << 13, 1 << 17]
    x = inputs.complex_signals(1, sum(lengths), seed=707)[0]
    gy = None
    plan = _lib.Plan(lengths, len(lengths), graph=True, seg_log=seg_log, streams=streams,
                     opts={"tile_first": True, "tile_split": split})
    assert plan.opts()["tile_split"] == split
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    gx = torch.empty(plan.in_elems, dtype=torch.complex64, device="cuda")
    gy = inputs.complex_signals(1, plan.out_elems, seed=708)[0]
    gyt = torch.from_numpy(gy).cuda()
    sp = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        y.fill_(float("nan"))
        gx.fill_(float("nan"))
        plan.forward(xt.data_ptr(), y.data_ptr(), sp)
        plan.adjoint(gyt.data_ptr(), gx.data_ptr(), sp)
    torch.cuda.synchronize()
    plan.status_poll()
    ys = split_out(y.cpu().numpy(), lengths)
    gxs = split_in(gx.cpu().numpy(), lengths)
    gys = split_out(gy, lengths)
    for s, xs in enumerate(split_in(x, lengths)):
        check_forward_levels(ys[s], oracle.forward(xs.astype(np.complex128)), xs, f"split={split} s={s}")
        check_adjoint(gxs[s], oracle.adjoint(gys[s].astype(np.complex128)), gys[s], f"split={split} s={s}")


@pytest.mark.parametrize("seg_log,streams,early", [(14, 3, False), (16, 1, True), (18, 4, False)])
def test_top_overlap(oracle, seg_log, streams, early):
    """top_overlap: the cols passes of the levels above the segment size run on
    their own stream, each level's rows pass waiting only for its own cols pass
    (alone: from the end of the segments; with top_cols_early: from the start)
    -- under graph replay, repeated, every level of every signal."""
    lengths = [1 << 20, 1 << 17, 1 << 19, 1 << 13]
    x = inputs.complex_signals(1, sum(lengths), seed=809)[0]
    plan = _lib.Plan(lengths, len(lengths), graph=True, seg_log=seg_log, streams=streams,
                     opts={"top_overlap": True, "top_cols_early": early})
    o = plan.opts()
    assert o["top_overlap"] is True and o["top_cols_early"] is early
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for _ in range(3):
            y.fill_(float("nan"))
            plan.forward(xt.data_ptr(), y.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    plan.status_poll()
    ys = split_out(y.cpu().numpy(), lengths)
    for k, xs in enumerate(split_in(x, lengths)):
        check_forward_levels(ys[k], oracle.forward(xs.astype(np.complex128)), xs, f"overlap seg={seg_log} s={k}")


@pytest.mark.parametrize("seg_log,streams", [(14, 3), (16, 1), (18, 4)])
def test_top_cols_early(oracle, seg_log, streams):
    """top_cols_early: the cols passes of the levels above the segment size run
    on their own stream during the segments, each into its own scratch, and
    their rows passes at the end -- under graph replay, repeated."""
    lengths = [1 << 20, 1 << 17, 1 << 19, 1 << 13]
    x = inputs.complex_signals(1, sum(lengths), seed=808)[0]
    plan = _lib.Plan(lengths, len(lengths), graph=True, seg_log=seg_log, streams=streams,
                     opts={"top_cols_early": True})
    assert plan.opts()["top_cols_early"] is True
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        y.fill_(float("nan"))
        plan.forward(xt.data_ptr(), y.data_ptr(), sp)
    torch.cuda.synchronize()
    plan.status_poll()
    ys = split_out(y.cpu().numpy(), lengths)
    for s, xs in enumerate(split_in(x, lengths)):
        check_forward_levels(ys[s], oracle.forward(xs.astype(np.complex128)), xs, f"early S={seg_log} s={s}")
