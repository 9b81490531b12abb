"""The table-driven FP64 exp/log used by the Jacobian kernels (Tang's methods) against CUDA's own
exp/log: at most 2 ulp apart over the whole fast range, and identical on the library path."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ulp_diff(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    ia = np.where(ia < 0, np.int64(-0x8000000000000000) - ia, ia)
    ib = np.where(ib < 0, np.int64(-0x8000000000000000) - ib, ib)
    return np.abs(ia - ib)


def test_fast_exp_log_within_two_ulp_of_cuda():
    from paper_1605_03262_b300 import build as pjbuild
    lib = ctypes.CDLL(pjbuild.build_calib())
    rng = np.random.default_rng(0)
    xe = np.concatenate([rng.uniform(-700, 700, 400000), rng.uniform(-1, 1, 200000), rng.uniform(-1e-6, 1e-6, 10000),
                         np.array([0.0, -0.0, 1.0, -1.0, 699.9, -699.9, 700.0, -700.0, 710.0, -750.0, np.inf, -np.inf])])
    xl = np.concatenate([10.0 ** rng.uniform(-300, 300, 400000), rng.uniform(0.5, 2.0, 200000),
                         1.0 + rng.uniform(-1e-6, 1e-6, 10000),
                         np.array([1.0, 2.0, 0.5, 1e-310, 0.0, -1.0, np.inf, 1.7976931348623157e308])])
    for x, which in ((xe, "exp"), (xl, "log")):
        xd = torch.as_tensor(x, dtype=torch.float64, device="cuda")
        outs = [torch.empty_like(xd) for _ in range(4)]
        rc = lib.pjc_fastmath_check(ctypes.c_void_p(xd.data_ptr()), ctypes.c_int(len(x)),
                                    *[ctypes.c_void_p(o.data_ptr()) for o in outs])
        assert rc == 0
        ef, el, lf, ll = (o.cpu().numpy() for o in outs)
        f, ref = (ef, el) if which == "exp" else (lf, ll)
        finite = np.isfinite(ref)
        assert np.array_equal(np.isnan(f), np.isnan(ref))
        assert np.array_equal(f[~finite & ~np.isnan(ref)], ref[~finite & ~np.isnan(ref)])
        nz = finite & (ref != 0)
        assert _ulp_diff(f[nz], ref[nz]).max() <= 2, which
        assert np.array_equal(f[finite & (ref == 0)], ref[finite & (ref == 0)])
