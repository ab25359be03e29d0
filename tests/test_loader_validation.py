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
