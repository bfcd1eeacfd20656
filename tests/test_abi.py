"""The C-ABI library builds, loads and exports every symbol include/mockskewer.h
declares; argument validation works without touching a GPU."""
import ctypes as C
import os
import re

import pytest

import paper_2310_18996_gb300 as mk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mockskewer.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mk_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = mk.lib()
    decl = declared_symbols()
    assert len(decl) >= 12
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(mk.EXPORTS) == decl


def test_struct_layouts_match_header_sizes():
    # 4 doubles, 4 int32, a pointer, interp and p_s_nodes (int32), a pointer
    assert C.sizeof(mk.SkewerParams) == 8 * 4 + 4 * 4 + 8 + 4 + 4 + 8
    assert C.sizeof(mk.FgpaNodes) == 8 + 4 * 8 * mk.MAX_NODES
    assert mk.QSO_DTYPE.itemsize == 32
    assert C.sizeof(mk.StatsOut) == 8 * (32 * 10 + 32 * 64 * 3 + 32 * 5)


def test_null_arguments_are_rejected_without_a_device():
    L = mk.lib()
    assert L.mk_create(None, 0, None, None) == mk.MK_EINVAL
    h = C.c_void_p()
    assert L.mk_create(C.byref(h), 0, None, None) == mk.MK_EINVAL
    assert not h.value
    assert L.mk_sync(None) == mk.MK_EINVAL
    assert L.mk_set_stream(None, None) == mk.MK_EINVAL
    assert L.mk_load_box(None, None, None, None, None) == mk.MK_EINVAL
    assert L.mk_last_error(None) == b"no context"
    L.mk_destroy(None)
    L.mk_free_box(None)


def test_context_creation_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = mk.lib()
    h = C.c_void_p()
    cos = mk.Cosmo(omega_m=0.3147, lambda_lya=1215.67)
    assert L.mk_create(C.byref(h), 0, None, C.byref(cos)) == mk.MK_ECUDA
    assert not h.value
    with pytest.raises(RuntimeError):
        mk.Context()


# ------------------------------------------------------------ Sec. 2.6 host logic
def test_ps_tune_report_layout():
    assert C.sizeof(mk.PsTuneReport) == 8 + 8 + 8 + 3 * 8 * 32 + 3 * 8 + 8 * mk.PS_TUNE_MAX_PASSES


@pytest.mark.parametrize("a,s", [(0.3, 0.8), (1.2, 1.6), (0.08, 2.4), (2.0, 3.0), (0.02, 3.5), (0.7, 0.0)])
def test_gauss_moments_match_oracle(a, s):
    from oracle import ps_tuning
    f, sf = mk.fgpa_gauss_moments(a, s)
    fo, sfo = ps_tuning.fgpa_gauss_moments(a, s)
    assert abs(f - fo) < 1e-13 and abs(sf - sfo) < 1e-12


@pytest.mark.parametrize("fbar,frac", [(0.95, 0.2), (0.8, 0.5), (0.55, 0.7), (0.3, 0.9), (0.9, 0.05)])
def test_fit_a_bsigma_matches_oracle(fbar, frac):
    from oracle import ps_tuning
    sf = frac * (fbar * (1 - fbar)) ** 0.5
    a, s = mk.fit_a_bsigma(fbar, sf)
    ao, so = ps_tuning.fit_a_bsigma(fbar, sf)
    assert abs(a / ao - 1) < 1e-8 and abs(s / so - 1) < 1e-8


def test_fit_a_bsigma_rejects_unreachable_targets():
    for fbar, sf in ((0.8, 0.4), (1.0, 0.1), (0.5, 0.0), (0.0, 0.1)):
        with pytest.raises(mk.MkError):
            mk.fit_a_bsigma(fbar, sf)
    with pytest.raises(mk.MkError):
        mk.fgpa_gauss_moments(-1.0, 0.5)
