"""pj_batch_run_noalloc: the batched launch for callers that cannot allocate device memory (for
example a solver with a fixed memory pool that forbids cudaMalloc/cudaFree inside its time step).
Called through the C ABI twice in a row with new inputs, its Jacobians must match the existing
plain entry point; more items than its static scratch holds must be rejected with a clear error.
This file is collected last on purpose."""
import ctypes

import numpy as np
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


def _close(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return bool(np.all(np.abs(a - b) <= 1e-10 * np.maximum(np.abs(b), 1e-20)))


def test_noalloc_batched_launch_matches_plain_launch_on_two_calls():
    pj, fn = _fn()
    models = [synth.config_model(0), synth.config_model(1), mechs.mixed_model(seed=41, n_species=17, n_reactions=90)]
    gms = [pj.Model(synth.to_bytes(m)) for m in models]
    sizes = [700, 1100, 257]
    stream = torch.cuda.current_stream()
    for call in range(2):
        items = (pj.pj_batch_item * len(gms))()
        keep = []
        for k, (g, n) in enumerate(zip(gms, sizes)):
            T, P, Y = (torch.as_tensor(a, device="cuda") for a in synth.generate_states(g.n_species, n, seed=10 * call + k))
            N = g.n_species
            J = torch.full((n, N + 1, N + 1), float("nan"), dtype=torch.float64, device="cuda")
            keep.append((g, T, P, Y, J))
            it = items[k]
            it.mech, it.n = g.handle, n
            it.T, it.P, it.Y, it.ldy = T.data_ptr(), P.data_ptr(), Y.data_ptr(), N
            it.jac, it.ldj, it.dydt, it.ldd = J.data_ptr(), (N + 1) ** 2, None, 0
        rc = fn(items, len(gms), 0, 0, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, pj.library().pj_last_error()
        torch.cuda.synchronize()
        for g, T, P, Y, J in keep:
            assert _close(J, g.eval_jacobian(T, P, Y))


def test_noalloc_rejects_more_items_than_its_scratch_holds():
    pj, fn = _fn()
    g = pj.Model(synth.to_bytes(synth.config_model(0)))
    items = (pj.pj_batch_item * 65)()
    for it in items:
        it.mech, it.n, it.ldy, it.ldj = g.handle, 0, g.n_species, (g.n_species + 1) ** 2
    rc = fn(items, 65, 0, 0, None)
    assert rc == -1
    assert b"64" in pj.library().pj_last_error()
