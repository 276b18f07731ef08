"""CPU checks of the C-ABI library: it loads, exports every function that
include/tmr.h declares, and its host-only entry points behave."""
import ctypes

import pytest


def test_library_exports_every_declared_symbol():
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    names = tmr.header_symbols()
    assert len(names) >= 12
    raw = ctypes.CDLL(tmr.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_default_options_and_errors_without_device():
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    o = tmr.tmr_default_options()
    assert (o.m, o.init, o.power_iters, o.phase_iters) == (5, tmr.TMR_INIT_SPECTRAL, 100, 100)
    assert o.clip == 2.0 and o.tol == 0.0
    o2 = tmr.tmr_default_options(init="bp", m=3)
    assert (o2.init, o2.m) == (tmr.TMR_INIT_BP, 3)
    import numpy as np
    with pytest.raises(tmr.TMRError):
        tmr.tmr_create(64, 4, 4, np.ones(4 * 64, np.complex64), opt=dict(m=0))
    with pytest.raises(TypeError):
        tmr.tmr_create(64, 4, 4, np.ones(4 * 64, np.complex128))
    tmr.lib.tmr_destroy(None)  # NULL is allowed


def test_header_documents_every_entry_point():
    tmr = pytest.importorskip("paper_2302_13524_gb300")
    text = open(tmr._lib.HEADER).read()
    for n in tmr.header_symbols():
        assert text.count(n) >= 1
    for sec in ("Eq. optTMsmall2", "Eq. derivative", "Eq. optphase", "Eq. phaseoffset"):
        assert sec in text
