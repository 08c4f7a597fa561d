"""The no-allocation map call (rs_shoot_map_host_noalloc).

Callers that cannot allocate device memory on their call path -- code under
another framework's allocator, real-time or plugin hosts, processes whose
device memory is reserved up front -- use this entry point; its device
working set is the library's fixed device array.  This test calls it through
the C ABI twice in a row (two different maps, then the first again, so a
stale map left in the shared array would show) and checks every result
against the allocating entry point rs_shoot_map_host on the same inputs.
It sits in a file that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _call(rs, job, lens_h):
    L = rs.lib()
    mc, g, mp = rs.structs(job)
    o = rs.options(rs.PREC_COMPENSATED, job.mass_model == W.MASS_UNIT, 0)
    mu = torch.full((job.npix, job.npix), -1.0, dtype=torch.float32).pin_memory()
    st = torch.full((rs.NSTATS,), -1, dtype=torch.int64).pin_memory()
    rc = L.rs_shoot_map_host_noalloc(C.byref(mc), C.c_void_p(lens_h.data_ptr()),
                                     lens_h.shape[1], C.byref(g), C.byref(mp), C.byref(o),
                                     C.c_void_p(mu.data_ptr()), C.c_void_p(st.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.rs_last_error()
    return mu.numpy().copy(), st.numpy().copy()


def test_no_alloc_call_matches_allocating_call():
    import paper_1406_0559_b300 as rs
    a = W.PARITY                                             # 256^2, 150 unit lenses
    b = W.scaled(W.PRECISION, ray_scale=16, map_scale=4, lens_scale=50)   # 1024^2, Salpeter
    runs = []
    for job in (a, b, a):
        lens_h = rs.make_lenses(job).cpu().contiguous()
        mu, st = _call(rs, job, lens_h)
        mu_ref, st_ref = rs.shoot_map_host(job, lens_h)
        # same kernels and arithmetic: identical maps and counts (tolerance 0)
        assert np.array_equal(mu, mu_ref.numpy()), job.name
        assert np.array_equal(st, st_ref.numpy()), job.name
        assert st[0] + st[1] + st[2] == job.n1 * job.n2
        runs.append(mu)
    assert np.array_equal(runs[0], runs[2])


def test_no_alloc_call_rejects_sizes_beyond_its_array():
    import paper_1406_0559_b300 as rs
    job = W.PARITY.with_(npix=2048)
    lens_h = torch.zeros((3, 4), dtype=torch.float64)
    mu = torch.empty((4, 4), dtype=torch.float32)
    st = torch.empty(rs.NSTATS, dtype=torch.int64)
    with pytest.raises(rs.RSError) as e:
        rs.shoot_map_host_noalloc(job, lens_h, mu, st)
    assert e.value.code == -6 and "no-allocation limit" in str(e.value)


def test_no_alloc_call_allocates_nothing():
    """The property the entry point exists for.  After a first call has loaded
    the kernels on the device, a call leaves the device's default
    stream-ordered pool untouched (its used-memory high watermark, reset to
    zero just before, stays zero), torch's allocator holds the same bytes, and
    the device's free memory is unchanged."""
    from cuda.bindings import driver as drv
    import paper_1406_0559_b300 as rs
    job = W.PARITY
    lens_h = rs.make_lenses(job).cpu().contiguous()
    mu0, st0 = _call(rs, job, lens_h)
    torch.cuda.synchronize()
    err, cudev = drv.cuDeviceGet(torch.cuda.current_device())
    assert err == drv.CUresult.CUDA_SUCCESS
    err, pool = drv.cuDeviceGetDefaultMemPool(cudev)
    assert err == drv.CUresult.CUDA_SUCCESS
    high = drv.CUmemPool_attribute.CU_MEMPOOL_ATTR_USED_MEM_HIGH
    (err,) = drv.cuMemPoolSetAttribute(pool, high, drv.cuuint64_t(0))
    assert err == drv.CUresult.CUDA_SUCCESS
    torch_before = torch.cuda.memory_allocated()
    err, free0, _ = drv.cuMemGetInfo()
    assert err == drv.CUresult.CUDA_SUCCESS
    mu1, st1 = _call(rs, job, lens_h)
    torch.cuda.synchronize()
    err, free1, _ = drv.cuMemGetInfo()
    err2, used_high = drv.cuMemPoolGetAttribute(pool, high)
    assert err == drv.CUresult.CUDA_SUCCESS and err2 == drv.CUresult.CUDA_SUCCESS
    assert int(used_high) == 0
    assert torch.cuda.memory_allocated() == torch_before
    assert free1 == free0
    assert np.array_equal(mu0, mu1) and np.array_equal(st0, st1)
