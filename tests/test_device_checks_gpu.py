"""Device-side work-item checks and graph-cache bookkeeping, through the C ABI.

A kernel given a work item that does not describe part of a planned signal
must skip it and raise MRDFT_EDEVICE in the plan's status word, and the plan
must work again once the item is restored.  The planted items below are
chosen so that every access they would cause still lies inside the plan's
buffers (the neighbouring signal's data), so that a missing check shows up
as a wrong result, never as a memory fault.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1507_02525_gb300 import _lib, inputs  # noqa: E402

from tests._parity import check_adjoint, check_forward_levels  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _items(plan, lst):
    out, k = [], 0
    while True:
        v = plan.debug_item(lst, k)
        if v is None:
            return out
        out.append(v)
        k += 1


def _fwd(plan, x):
    xt = torch.from_numpy(x.reshape(-1)).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y


def _adj(plan, g):
    gt = torch.from_numpy(g.reshape(-1)).cuda()
    gx = torch.empty(plan.in_elems, dtype=torch.complex64, device="cuda")
    plan.adjoint(gt.data_ptr(), gx.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return gx


N, M = 1 << 16, 16


@pytest.mark.parametrize("which", ["level15", "tile"])
def test_planted_item_is_skipped_and_reported(oracle, which):
    x = inputs.complex_signals(2, N, seed=500)
    g = inputs.targets(2, N, seed=501)
    plan = _lib.Plan([N], 2)
    if which == "level15":
        # a level-15 item of signal 0 (window 1, block 1 exist only at level 15)
        lst = 1
        idx = next(k for k, v in enumerate(_items(plan, 1)) if v[0] == 0 and v[1] == 1 and v[2] == 1)
        old = plan.debug_item(lst, idx)
        bad = [0, 2, 1, 0]            # window 2 does not exist at level 15 of a 2^16 signal
    else:
        lst = 0
        # signal 0's last tile (signal 0 is listed first); tile 16 would read
        # signal 1's input and write signal 0's level 2 if it were not checked
        idx = next(k for k, v in enumerate(_items(plan, 0)) if v[2] == 15)
        old = plan.debug_item(lst, idx)
        assert old[0] == 0 and old[1] == (1 | (12 << 16))
        bad = [old[0], old[1], 16, 0]  # tile 16 of a signal of 16 tiles
    plan.debug_item(lst, idx, bad)
    _fwd(plan, x)
    with pytest.raises(_lib.MrdftError) as e:
        plan.status_poll()
    assert e.value.status == _lib.MRDFT_EDEVICE
    _adj(plan, g)
    with pytest.raises(_lib.MrdftError) as e:
        plan.status_poll()
    assert e.value.status == _lib.MRDFT_EDEVICE
    plan.status_poll()  # cleared by the previous poll
    plan.debug_item(lst, idx, old)
    y = _fwd(plan, x).cpu().numpy().reshape(2, M, N)
    gx = _adj(plan, g).cpu().numpy().reshape(2, N)
    plan.status_poll()
    for s in range(2):
        check_forward_levels(y[s], oracle.forward(x[s].astype(np.complex128)), x[s], f"restored s={s}")
        check_adjoint(gx[s], oracle.adjoint(g[s].astype(np.complex128)), g[s], f"restored s={s}")


def test_debug_item_bounds():
    plan = _lib.Plan([N], 2)
    n_lv = len(_items(plan, 1))
    assert n_lv > 0 and plan.debug_item(1, n_lv) is None and plan.debug_item(1, -1) is None
    assert len(_items(plan, 0)) == 2 * N // 4096


def test_graph_cache_is_bounded():
    """New output buffers on every call: the plan keeps at most 4 executable
    graphs per direction and re-targets the oldest one past that."""
    B = 2
    x = torch.from_numpy(inputs.complex_signals(B, 1 << 15, seed=7).reshape(-1)).cuda()
    plan = _lib.Plan([1 << 15], B, graph=True)
    sp = torch.cuda.current_stream().cuda_stream
    ref = None
    keep = []  # every output stays allocated, so that each call sees a new address
    for k in range(10):
        y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
        keep.append(y)
        plan.forward(x.data_ptr(), y.data_ptr(), sp)
        torch.cuda.synchronize()
        if ref is None:
            ref = y.clone()
        assert torch.equal(y, ref), k
        st = plan.graph_stats()
        assert st["cached"] <= 4, st
    st = plan.graph_stats()
    assert st["captures"] == 10 and st["updates"] == 6, st
    plan.status_poll()
