"""Host-side validation of ck_load_mechanism, which runs before any CUDA call
and so needs no GPU: a malformed description is refused with CK_EINVAL and a
message naming the problem."""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism
from synth.handmade import cyclic_network

ck = pytest.importorskip("paper_1608_05794_gb300.ck")


def _refused(m, match, **kw):
    with pytest.raises(ck.CKError) as e:
        ck.load_mechanism(m, **kw)
    msg = str(e.value)
    assert "invalid argument" in msg or "size beyond" in msg, msg
    assert match in msg, msg


def _copy(m):
    return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}


def test_reactor_type_must_be_0_or_1():
    _refused(cyclic_network(), "reactor", reactor=2)


def test_explicit_reverse_needs_its_coefficients():
    m = _copy(cyclic_network())
    m["rev"][0] = 2
    _refused(m, "arrh_rev")
    m["arrh_rev"] = np.zeros((len(m["rev"]), 3))
    _refused(m, "reverse A must be positive")


def test_reversible_flag_range():
    m = _copy(cyclic_network())
    m["rev"] = np.full(len(m["rev"]), 3, np.uint8)
    _refused(m, "reversible must be 0, 1 or 2")


def test_species_index_and_padding():
    m = _copy(cyclic_network())
    m["reac"][0, 0] = 99
    _refused(m, "species index out of range")
    m = _copy(cyclic_network())
    m["prod"][0] = [-1, 1, -1]
    _refused(m, "padding must come last")


def test_arrhenius_and_falloff_parameters():
    m = _copy(cyclic_network())
    m["arrh"][2, 0] = -1.0
    _refused(m, "Arrhenius A must be positive")
    m = _copy(cyclic_network())
    m["arrh0"][4, 0] = 0.0  # reaction 4 is the Lindemann one
    _refused(m, "low-pressure A must be positive")


def test_atom_balance_is_checked():
    m = _copy(load_mechanism(CONFIGS["small"]["mech"]))
    # swap a product for a species of another composition
    r = 0
    sp = int(m["prod"][r, 0])
    other = next(k for k in range(len(m["mw"])) if not np.array_equal(m["elem"][k], m["elem"][sp]))
    m["prod"][r, 0] = other
    _refused(m, "atom-balanced")


def test_molar_masses_must_be_positive():
    m = _copy(cyclic_network())
    m["mw"] = m["mw"].copy()
    m["mw"][1] = -1.0
    _refused(m, "mw must be positive")


# argument checks of other entry points that also come before any CUDA call
CK_EINVAL, CK_ERANGE = 1, 6


def test_lu_entry_points_check_their_sizes():
    L = ck._lib
    buf = np.zeros(16)
    ip = np.zeros(16, np.int32)
    for dim in (0, 129):
        assert L.ck_lu_factor(1, dim, buf.ctypes.data, ip.ctypes.data, ip.ctypes.data, None) == CK_ERANGE
        assert L.ck_lu_solve(1, dim, buf.ctypes.data, ip.ctypes.data, buf.ctypes.data, None) == CK_ERANGE
    assert L.ck_lu_factor(-1, 4, buf.ctypes.data, ip.ctypes.data, ip.ctypes.data, None) == CK_ERANGE
    assert L.ck_lu_factor(0, 4, None, None, None, None) == 0  # empty batch: nothing to do
    assert L.ck_lu_factor(1, 4, None, ip.ctypes.data, ip.ctypes.data, None) == CK_EINVAL


def test_group_and_server_arguments():
    import ctypes as C
    L = ck._lib
    groups = (ck.Group * 1)()
    assert L.ck_integrate_groups(5, 1, groups, 0, None) == CK_EINVAL   # method
    assert L.ck_integrate_groups(0, 0, groups, 0, None) == CK_ERANGE   # n_groups
    assert L.ck_integrate_groups(0, 17, groups, 0, None) == CK_ERANGE
    assert L.ck_integrate_groups(0, 1, None, 0, None) == CK_EINVAL
    out = C.c_void_p()
    assert L.ck_server_create(0, 4, 0, C.byref(out)) == CK_EINVAL       # budget
    assert L.ck_server_create(1 << 30, 0, 0, C.byref(out)) == CK_ERANGE  # streams
    assert L.ck_server_create(1 << 30, 65, 0, C.byref(out)) == CK_ERANGE


def test_integrating_entry_points_refuse_batches_beyond_the_queue_limit():
    # a 32-bit device work queue hands out reactors; n above CK_MAX_REACTORS
    # (2^30) is refused with CK_ERANGE before any handle or pointer is used
    import ctypes as C
    L = ck._lib
    n = (1 << 31) - 1
    for fn in (L.ck_integrate_ros4, L.ck_integrate_rkf45, L.ck_integrate_ros4_noalloc):
        assert fn(None, n, None, None, None, None, None, None, None, None) == CK_ERANGE
        assert "MAX_REACTORS" in L.ck_last_error().decode()
        assert fn(None, (1 << 30) + 1, None, None, None, None, None, None, None, None) == CK_ERANGE
    groups = (ck.Group * 1)()
    groups[0].n = n
    assert L.ck_integrate_groups(0, 1, groups, 0, None) == CK_ERANGE
    t = C.c_uint64()
    assert L.ck_submit(None, None, 0, n, None, None, None, None, None, None, C.byref(t)) == CK_ERANGE
