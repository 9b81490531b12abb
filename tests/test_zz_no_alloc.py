"""pj_batch_run_noalloc: the batched launch for callers that cannot allocate device memory where
they call the library (for example a reacting-flow solver with a fixed device memory pool that
forbids cudaMalloc/cudaFree inside its time step, or code that must not meet an allocation
failure mid-run). Its only device scratch is the tile counter in a static array of the library.

Called through the C ABI twice in a row with new inputs, its Jacobians (with and without the
source terms beside them) and its source terms must equal, bit for bit, those of the plain
per-model entry points; an item without states may sit between others; a second call must leave
the device's free memory unchanged; the call must not wait on the host for earlier work on its
stream; more items than one call's table holds must be rejected with a clear error.

This file is collected last on purpose: the static array is shared by every call in the process
and keeps the last call's contents, so these tests also show that a call is correct after
whatever the earlier tests left in it (they pass run alone in a fresh process as well).
"""
import ctypes
import time

import pytest

from paper_1605_03262_b300 import synth
from tests import mechs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fn():
    import paper_1605_03262_b300 as pj
    fn = pj.library().pj_batch_run_noalloc
    fn.argtypes = [ctypes.POINTER(pj.pj_batch_item), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return pj, fn


def _models(pj):
    models = [synth.config_model(0), synth.config_model(1), mechs.mixed_model(seed=41, n_species=17, n_reactions=90)]
    return [pj.Model(synth.to_bytes(m)) for m in models]


def _items(pj, gms, sizes, which, with_dydt, seed):
    """The C item array and the tensors behind it; outputs start as NaN."""
    items = (pj.pj_batch_item * len(gms))()
    keep = []
    for k, (g, n) in enumerate(zip(gms, sizes)):
        N = g.n_species
        T, P, Y = (torch.as_tensor(a, device="cuda") for a in synth.generate_states(N, max(n, 1), seed=seed + k))
        T, P, Y = T[:n].contiguous(), P[:n].contiguous(), Y[:n].contiguous()
        J = torch.full((n, N + 1, N + 1), float("nan"), dtype=torch.float64, device="cuda") if which == 0 else None
        F = torch.full((n, N + 1), float("nan"), dtype=torch.float64, device="cuda") if (which == 1 or with_dydt) \
            else None
        keep.append((g, T, P, Y, J, F))
        it = items[k]
        it.mech, it.n = g.handle, n
        it.T, it.P, it.Y, it.ldy = T.data_ptr(), P.data_ptr(), Y.data_ptr(), N
        it.jac, it.ldj = (J.data_ptr(), (N + 1) ** 2) if J is not None else (None, 0)
        it.dydt, it.ldd = (F.data_ptr(), N + 1) if F is not None else (None, 0)
    return items, keep


def _check_against_plain(keep, which):
    for g, T, P, Y, J, F in keep:
        if T.numel() == 0:
            continue
        if which == 0:
            if F is None:
                assert torch.equal(J, g.eval_jacobian(T, P, Y))
            else:
                Jp, Fp = g.eval_jacobian(T, P, Y, dydt=True)
                assert torch.equal(J, Jp)
                assert torch.equal(F, Fp)
        else:
            assert torch.equal(F, g.eval_dydt(T, P, Y))


@pytest.mark.parametrize("which,with_dydt", [(0, False), (0, True), (1, False)],
                         ids=["jacobian", "jacobian+dydt", "dydt"])
def test_noalloc_batched_launch_equals_plain_launch_on_two_calls(which, with_dydt):
    pj, fn = _fn()
    gms = _models(pj)
    stream = torch.cuda.current_stream()
    # the second call has an item without states between two others
    for call, sizes in enumerate(([700, 1100, 257], [313, 0, 129])):
        items, keep = _items(pj, gms, sizes, which, with_dydt, seed=100 * call + 10 * which)
        rc = fn(items, len(gms), which, 0, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, pj.library().pj_last_error()
        torch.cuda.synchronize()
        _check_against_plain(keep, which)


def test_noalloc_second_call_leaves_free_device_memory_unchanged():
    pj, fn = _fn()
    gms = _models(pj)
    stream = torch.cuda.current_stream()
    items, keep = _items(pj, gms, [300, 200, 100], 0, True, seed=7)
    assert fn(items, len(gms), 0, 0, ctypes.c_void_p(stream.cuda_stream)) == 0   # warm-up (module load)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert fn(items, len(gms), 0, 0, ctypes.c_void_p(stream.cuda_stream)) == 0, pj.library().pj_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check_against_plain(keep, 0)


def test_noalloc_call_does_not_wait_for_earlier_work_on_its_stream():
    pj, fn = _fn()
    gms = _models(pj)[:1]
    stream = torch.cuda.current_stream()
    items, keep = _items(pj, gms, [64], 0, False, seed=3)
    assert fn(items, 1, 0, 0, ctypes.c_void_p(stream.cuda_stream)) == 0
    torch.cuda.synchronize()
    torch.cuda._sleep(200_000_000)           # about 0.1 s of GPU time ahead of the call on the stream
    t0 = time.perf_counter()
    rc = fn(items, 1, 0, 0, ctypes.c_void_p(stream.cuda_stream))
    dt = time.perf_counter() - t0
    pending = not stream.query()
    torch.cuda.synchronize()
    assert rc == 0, pj.library().pj_last_error()
    assert pending and dt < 0.05
    _check_against_plain(keep, 0)


def test_noalloc_rejects_more_items_than_its_table_holds():
    pj, fn = _fn()
    g = pj.Model(synth.to_bytes(synth.config_model(0)))
    items = (pj.pj_batch_item * 65)()
    for it in items:
        it.mech, it.n, it.ldy, it.ldj = g.handle, 0, g.n_species, (g.n_species + 1) ** 2
    rc = fn(items, 65, 0, 0, None)
    assert rc == -1
    assert b"64" in pj.library().pj_last_error()
