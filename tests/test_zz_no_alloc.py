"""The allocation-free operator entry point (wt_apply_operator_static).

Callers that cannot allocate device memory (a host framework's memory pool,
an embedded solver that only receives buffers) use this entry point: it
keeps every temporary in one static device array.  The test calls it through
the C ABI and checks it against the ordinary wt_apply_operator on two calls
in a row (the second call reuses the scratch left by the first).  It lives
in its own file, collected last, and passes alone or after the other tests.
"""

import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case(Nx, Nz, L, seed):
    r = np.random.default_rng(seed)
    x = np.arange(Nx) * L / Nx
    h = 1.0 - 0.3 * np.exp(-((x - L / 2) / (L / 8)) ** 2)
    ea = 0.05 * np.cos(2 * np.pi * x / L + r.uniform())
    eb = ea + 0.001 * r.standard_normal(Nx)
    p = r.standard_normal((Nz + 1, 1, Nx))
    return h, ea, eb, p


def test_static_operator_matches_wt_apply_operator_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    lib = w.lib
    f = lib.wt_apply_operator_static
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double] + [ctypes.c_void_p] * 6
    f.restype = ctypes.c_int
    dev = torch.device("cuda", 0)
    for call, (Nx, Nz, L, seed) in enumerate([(1024, 24, 32.0, 1), (256, 16, 2 * math.pi, 2)]):
        h, ea, eb, p = _case(Nx, Nz, L, seed)
        T = w.Tank(Nx, 1, Nz, L, h[None])
        ref = T.apply_operator(ea[None], eb[None], np.ascontiguousarray(p), w.WT_FP64)
        T.close()
        th, tea, teb, tp = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (h, ea, eb, p))
        tAp = torch.full_like(tp, float("nan"))
        torch.cuda.synchronize()
        st = f(Nx, Nz, L, th.data_ptr(), tea.data_ptr(), teb.data_ptr(), tp.data_ptr(), tAp.data_ptr(), None)
        assert st == w.WT_OK, w.wt_last_error()
        got = tAp.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), call
    # sizes beyond the static array are rejected with a clear error
    tp = torch.zeros((33, 1, 4096), dtype=torch.float64, device=dev)
    ts = torch.ones(4096, dtype=torch.float64, device=dev)
    st = f(4096, 32, 1.0, ts.data_ptr(), ts.data_ptr(), ts.data_ptr(), tp.data_ptr(), tp.data_ptr(), None)
    assert st == w.WT_EINVAL
    assert "2048" in w.wt_last_error()[1]
