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


@pytest.mark.parametrize("q,dt", [(19, "float64"), (27, "float32")])
def test_static_reduce_many_chunks_null_mask_side_stream(torch, q, dt):
    # 3 * 65536 + 123 cells: four partial sums, the last one over a ragged chunk, summed in a fixed
    # order; no mask; a device out and then a host out, both ordered on a side stream
    n = 3 * 65536 + 123
    rng = np.random.default_rng(123 + q)
    host = (1.0 / q + 0.01 * rng.standard_normal((q, n))).astype(dt)
    import oracle.oracle as O  # lattice vectors for the reference sums
    c = O.lattice(q)[0].astype(np.float64)
    h64 = host.astype(np.float64)
    ref = np.concatenate([[h64.sum()], c.T @ h64.sum(axis=1)])
    code = lbm.DTYPE_F64 if dt == "float64" else lbm.DTYPE_F32
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        f = torch.from_numpy(host).to("cuda", non_blocking=False)
        for call in range(2):
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lbm.lib().lbm_reduce_static(q, _ptr(f), code, None, n, _ptr(out), ctypes.c_void_p(side.cuda_stream))
            assert rc == 0, lbm.lib().lbm_reduce_static_error()
            side.synchronize()
            got = out.cpu().numpy()
            tol = 1e-12 * np.abs(h64).sum()
            assert np.abs(got - ref).max() <= tol, (call, got, ref)
            hout = np.full(4, np.nan)
            rc = lbm.lib().lbm_reduce_static(q, _ptr(f), code, None, n, hout.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.c_void_p(side.cuda_stream))
            assert rc == 0, lbm.lib().lbm_reduce_static_error()
            assert np.array_equal(hout, got)


def test_static_reduce_rejects_host_inputs(torch):
    f = torch.zeros(19 * 64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    host_mask = np.zeros(64, np.uint8)
    rc = lbm.lib().lbm_reduce_static(19, _ptr(f), lbm.DTYPE_F32, host_mask.ctypes.data_as(ctypes.c_void_p), 64,
                                     _ptr(out), None)
    assert rc == lbm.EINVAL
    assert b"mask" in lbm.lib().lbm_reduce_static_error()
    host_f = np.zeros(19 * 64, np.float32)
    rc = lbm.lib().lbm_reduce_static(19, host_f.ctypes.data_as(ctypes.c_void_p), lbm.DTYPE_F32, None, 64,
                                     _ptr(out), None)
    assert rc == lbm.EINVAL
    assert b"f must be device memory" in lbm.lib().lbm_reduce_static_error()
