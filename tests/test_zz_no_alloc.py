"""The allocation-free ROS4 entry point against the regular one.

ck_integrate_ros4_noalloc exists for callers that cannot let a library
allocate device memory, for example a CFD code that gives all device memory
to its own pool at start-up, or a process held to a fixed memory budget in
which an allocation in the middle of a time step could fail.  It keeps its
work-queue counter in a static device array instead of a per-call
allocation and keeps no Jacobian copies, so its results must equal those of
ck_integrate_ros4, and it must draw nothing from the device's memory pool.  This file
is collected last so that a stop at the first failure has already run every
other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism, reactor_states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


def _run(ck, fn, gm, p, y, dt):
    yd = torch.as_tensor(y.copy(), device="cuda")
    st = torch.empty(y.shape[0], dtype=torch.int32, device="cuda")
    steps = torch.empty((y.shape[0], 2), dtype=torch.int32, device="cuda")
    h = torch.zeros(y.shape[0], dtype=torch.float64, device="cuda")
    fn(gm, torch.as_tensor(p, device="cuda"), yd, torch.full((y.shape[0],), dt, dtype=torch.float64,
                                                              device="cuda"), st, h_inout=h, steps=steps)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), steps.cpu().numpy()


@pytest.mark.parametrize("name,n", [("small", 333), ("medium", 96)])
def test_noalloc_matches_regular_entry_point_twice(ck, name, n):
    cfg = CONFIGS[name]
    gm = ck.load_mechanism(load_mechanism(cfg["mech"]))
    y, p = reactor_states(name, n=n, seed_offset=41)
    ref_y, ref_st, ref_steps = _run(ck, ck.integrate_ros4, gm, p, y, cfg["dt"])
    for _ in range(2):  # two calls in a row share (and reset) the static counter
        y_na, st_na, steps_na = _run(ck, ck.integrate_ros4_noalloc, gm, p, y, cfg["dt"])
        assert np.array_equal(st_na, ref_st)
        assert np.max(np.abs(y_na[:, 0] - ref_y[:, 0]) / ref_y[:, 0]) <= 1e-6
        assert np.max(np.abs(y_na[:, 1:] - ref_y[:, 1:])) <= 1e-8
        assert np.array_equal(steps_na, ref_steps)
    assert np.all(ref_st == 0)


def _pool_used_high(reset=False):
    """High-water mark (bytes) of the current device's default stream-ordered
    memory pool, which every cudaMallocAsync of the library draws from; read
    through the driver API.  reset=True zeroes it first."""
    import ctypes as C
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int()
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    used_mem_high = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH
    v = C.c_uint64(0)
    if reset:
        assert cu.cuMemPoolSetAttribute(pool, used_mem_high, C.byref(v)) == 0
    assert cu.cuMemPoolGetAttribute(pool, used_mem_high, C.byref(v)) == 0
    return v.value


def test_noalloc_takes_no_pool_memory(ck):
    # the call draws nothing from the stream-ordered pool, while the regular
    # entry point (work-queue counter, Jacobian copies) does
    cfg = CONFIGS["medium"]
    gm = ck.load_mechanism(load_mechanism(cfg["mech"]))
    y, p = reactor_states("medium", n=64, seed_offset=43)
    _run(ck, ck.integrate_ros4_noalloc, gm, p, y, cfg["dt"])  # buffers of the helper itself come from torch
    torch.cuda.synchronize()
    _pool_used_high(reset=True)
    _run(ck, ck.integrate_ros4_noalloc, gm, p, y, cfg["dt"])
    assert _pool_used_high() == 0
    _run(ck, ck.integrate_ros4, gm, p, y, cfg["dt"])
    assert _pool_used_high() > 0


def test_noalloc_rejects_host_arrays_and_oversize_batches(ck):
    cfg = CONFIGS["small"]
    gm = ck.load_mechanism(load_mechanism(cfg["mech"]))
    y, p = reactor_states("small", n=4)
    st = np.zeros(4, np.int32)
    with pytest.raises(ck.CKError, match="device pointers only"):
        ck.integrate_ros4_noalloc(gm, np.ascontiguousarray(p), y.copy(), np.full(4, 1e-5), st)
    # a batch beyond the documented maximum is refused before anything runs
    rc = ck._lib.ck_integrate_ros4_noalloc(gm.h, (1 << 30) + 1, None, None, None, None, None, None, None,
                                           None)
    assert rc == 6  # CK_ERANGE
    assert "CK_NOALLOC_MAX_REACTORS" in ck._lib.ck_last_error().decode()
