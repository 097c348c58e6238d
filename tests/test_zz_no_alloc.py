"""The allocation-free reduction (lbm_reduce_static) against the context-based lbm_reduce.

lbm_reduce_static exists for callers that cannot let a library allocate device memory; it keeps its
partial sums in a static device array. This file is collected last so that, if it fails, a run
that stops at the first failure has already run every other test. It must pass both alone in a
fresh process and after the other tests (the static array keeps the previous call's contents).
"""
import ctypes

import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I

pytestmark = pytest.mark.gpu
lbm = pytest.importorskip("paper_2506_21804_gb300.lbm")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    lbm.lib()
    return t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("q,storage,rtol", [(19, lbm.F64, 1e-12), (27, lbm.F64, 1e-12), (19, lbm.F32, 1e-6)])
def test_static_reduce_matches_context_reduce_twice(torch, q, storage, rtol):
    # periodic box, no force, no inlet/outlet: lbm_reduce's sums equal the raw population moments
    w = I.random_box(40, 18, 11, seed=17, q=q, solid_frac=0.1, tau=0.7, cs=0.1)
    g = lbm.Lattice.from_workload(w, storage=storage)
    g.step(5)
    mass, mom = g.reduce()
    dt = torch.float64 if storage == lbm.F64 else torch.float32
    code = lbm.DTYPE_F64 if storage == lbm.F64 else lbm.DTYPE_F32
    f = torch.empty((q, w.N), dtype=dt, device="cuda")
    rc = lbm.lib().lbm_get_populations(g.h, _ptr(f), code)
    assert rc == 0
    mask = torch.from_numpy(np.ascontiguousarray(w.mask)).cuda()
    ref = np.array([mass, *mom])
    for call in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lbm.lib().lbm_reduce_static(q, _ptr(f), code, _ptr(mask), w.N, _ptr(out), None)
        assert rc == 0, lbm.lib().lbm_reduce_static_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - ref[0]) <= rtol * abs(ref[0]), (call, got, ref)
        assert np.abs(got[1:] - ref[1:]).max() <= rtol * abs(ref[0]), (call, got, ref)
        host = np.full(4, np.nan)
        rc = lbm.lib().lbm_reduce_static(q, _ptr(f), code, _ptr(mask), w.N, host.ctypes.data_as(ctypes.c_void_p), None)
        assert rc == 0, lbm.lib().lbm_reduce_static_error()
        assert np.array_equal(host, got)


def test_static_reduce_rejects_sizes_beyond_the_scratch(torch):
    f = torch.zeros(19 * 64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lbm.lib().lbm_reduce_static(19, _ptr(f), lbm.DTYPE_F32, None, (1 << 28) + 1, _ptr(out), None)
    assert rc == lbm.EINVAL
    assert b"outside" in lbm.lib().lbm_reduce_static_error()
