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


_FRESH = r"""
import math, sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
import paper_2406_00991_gb300 as w
from oracle import operator as op
Nx, Nz, L = 2048, 32, 64.0
r = np.random.default_rng(7)
g = op.Grid(Nx, 1, Nz, L)
h = 1.0 - 0.3 * np.exp(-((g.x - L / 2) / (L / 8)) ** 2)
ea = 0.05 * np.cos(2 * np.pi * g.x / L)
eb = ea + 0.001 * r.standard_normal(Nx)
p = r.standard_normal(g.shape)
ref = op.apply_A(g, op.Geometry(g, h, ea), op.Geometry(g, h, eb), p)
dev = torch.device("cuda", 0)
th, tea, teb, tp = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (h, ea, eb, p))
for call in range(2):
    tAp = torch.full_like(tp, float("nan"))
    torch.cuda.synchronize()
    st = w.wt_apply_operator_static(Nx, Nz, L, th, tea, teb, tp, tAp)
    assert st == w.WT_OK, w.wt_last_error()
    err = np.abs(tAp.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-11, (call, err)
print("fresh-process 2048x32 ok")
"""


def test_static_operator_largest_size_in_a_fresh_process():
    """The stated maximum (Nx = 2048, Nz = 32: the scratch layout's largest
    carve and the FP64 row pass that needs the dynamic shared-memory opt-in),
    called before any tank exists in the process, against the oracle's
    operator directly."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH % {"root": root}], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process 2048x32 ok" in r.stdout


def test_static_operator_rejects_sizes_and_host_memory():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2406_00991_gb300 as w
    dev = torch.device("cuda", 0)
    ts = torch.ones(2048, dtype=torch.float64, device=dev)
    tp = torch.zeros((34, 1, 2048), dtype=torch.float64, device=dev)
    assert w.wt_apply_operator_static(64, 33, 1.0, ts, ts, ts, tp, tp) == w.WT_EINVAL      # Nz > 32
    assert "32" in w.wt_last_error()[1]
    assert w.wt_apply_operator_static(96, 8, 1.0, ts, ts, ts, tp, tp) == w.WT_EINVAL       # not 2^k
    assert w.wt_apply_operator_static(64, 1, 1.0, ts, ts, ts, tp, tp) == w.WT_EINVAL       # Nz < 2
    host = np.ones(64)
    hp = np.zeros((9, 1, 64))
    assert w.wt_apply_operator_static(64, 8, 1.0, host, ts, ts, tp, tp) == w.WT_EINVAL
    assert w.wt_apply_operator_static(64, 8, 1.0, ts, ts, ts, tp, hp) == w.WT_EINVAL
    assert "device memory" in w.wt_last_error()[1]
