"""C-ABI library: builds for sm_103a, loads, exports every declared symbol,
and rejects invalid descriptors on the host (no GPU needed)."""
import ctypes

import pytest

from paper_1805_09498_gb300 import build, ffca


@pytest.fixture(scope="module")
def L():
    build.build()
    return ffca.lib()


def test_exports_every_declared_function(L):
    names = ffca.header_functions()
    assert "ffca_init" in names and "ffca_iterate" in names
    assert "ffca_loglik" in names and "ffca_wiener" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    assert ffca.ffca_status_str(0) == "ok"
    assert "singular" in ffca.ffca_status_str(4)
    assert ffca.ffca_status_str(99) == "unknown status"


def _desc(**kw):
    d = dict(I=3, J=3, F=4, N=10, ld=12, K=1, prec=1, y=None, v=None, lambda_=None, P=None,
             workspace=None, workspace_bytes=0, stream=None)
    d.update(kw)
    return ffca.ffca_desc(**d)


@pytest.mark.parametrize("kw,expect", [
    (dict(N=0), 1), (dict(ld=9), 1), (dict(ld=14), 1), (dict(K=0), 1), (dict(prec=2), 1),
    (dict(I=0), 1), (dict(J=0), 1), (dict(F=-1), 1), (dict(I=5), 7), (dict(J=7), 7),
    (dict(), 1),   # valid shape but null pointers
])
def test_init_rejects_bad_descriptors(L, kw, expect):
    ctx = ctypes.c_void_p()
    st = L.ffca_init(ctypes.byref(ctx), ctypes.byref(_desc(**kw)))
    assert st == expect
    assert not ctx.value


def test_workspace_size_zero_for_invalid(L):
    assert L.ffca_workspace_size(ctypes.byref(_desc(N=0))) == 0
    assert L.ffca_workspace_size(ctypes.byref(_desc(I=9))) == 0
    assert L.ffca_workspace_size(None) == 0


def test_null_context_is_an_argument_error(L):
    assert L.ffca_iterate(None, 1, None) == 1
    assert L.ffca_loglik(None, None) == 1
    assert L.ffca_wiener(None, None) == 1
    assert L.ffca_sync(None) == 1
    assert L.ffca_error_frequency(None) == -1
    assert L.ffca_set_p_update(None, 0, 0.0) == 1


def test_p_update_codes_match_the_header(L):
    """The binding's names of the updates of P carry the header's codes."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(ffca.__file__), "..", "include", "ffca.h")).read()
    codes = dict((m.group(1), int(m.group(2)))
                 for m in re.finditer(r"FFCA_P_(\w+) = (\d+)", hdr))
    assert codes == {k.upper(): v for k, v in ffca.P_UPDATES.items()}


def test_fault_injection_argument_checks(L):
    assert L.ffca_test_fault(None, 0) == 1
    assert L.ffca_test_fault(None, 1) == 1
