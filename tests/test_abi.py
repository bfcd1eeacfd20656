"""The C-ABI library builds, loads and exports every symbol include/mockskewer.h
declares; argument validation works without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
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


# ------------------------------------------------------------ Sec. 2.2 lognormal field (host)
def test_xi_and_lognormal_pk_match_oracle():
    from oracle import lognormal
    n = 1500
    dk = 6.0 / (n - 1)
    k = dk * np.arange(n)
    pk = np.where(k > 0, 80.0 * k ** 0.96 * np.exp(-(k / 1.5) ** 2), 0.0)
    r = np.array([0.0, 0.7, 5.0, 20.0, 80.0])
    np.testing.assert_allclose(mk.xi_of_pk(pk, dk, r), lognormal.xi_of_pk(pk, dk, r), rtol=1e-11, atol=1e-14)
    for B in (0.0, 0.3, 1.0):
        got = mk.lognormal_pk(pk, dk, B)
        ref = lognormal.lognormal_pk(pk, dk, B)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max() + 1e-300)
    # B large enough that 1 + B xi < 0 in a negative lobe of xi: both reject it
    xmin = lognormal.xi_of_pk(pk, dk, np.pi / (dk * (n - 1)) * np.arange(n)).min()
    assert xmin < 0
    with pytest.raises(ValueError):
        lognormal.lognormal_pk(pk, dk, -2.0 / xmin)
    for B in (-1.0, -2.0 / xmin):
        with pytest.raises(mk.MkError):
            mk.lognormal_pk(pk, dk, B)


# every ctypes structure of the binding and the C struct it mirrors
CTYPES_STRUCTS = {
    "mk_cosmo": mk.Cosmo, "mk_box_desc": mk.BoxDesc, "mk_skewer_params": mk.SkewerParams,
    "mk_fgpa_nodes": mk.FgpaNodes, "mk_stat_bins": mk.StatBins, "mk_stats_out": mk.StatsOut,
    "mk_surrogate_space": mk.SurrogateSpace, "mk_surrogate_norm": mk.SurrogateNorm,
    "mk_tune_target": mk.TuneTarget, "mk_tune_report": mk.TuneReport,
    "mk_qso_draw_params": mk.QsoDrawParams, "mk_ps_tune_report": mk.PsTuneReport,
}
NUMPY_RECORDS = {"mk_qso": mk.QSO_DTYPE, "mk_skewer": mk.SKEWER_DTYPE}


def test_binding_layouts_match_the_c_compiler(tmp_path):
    # sizeof and offsetof of every mirrored field, as gcc lays out the header
    # (plain C99), against the ctypes structures and numpy record dtypes
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    body, expect = [], []
    for cname, cls in CTYPES_STRUCTS.items():
        body.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(C.sizeof(cls))
        for f in cls._fields_:
            body.append(f'  printf("%zu\\n", offsetof({cname}, {f[0]}));')
            expect.append(getattr(cls, f[0]).offset)
    for cname, dt in NUMPY_RECORDS.items():
        body.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(dt.itemsize)
        for name in dt.names:
            body.append(f'  printf("%zu\\n", offsetof({cname}, {name}));')
            expect.append(dt.fields[name][1])
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"mockskewer.h\"\nint main(void) {\n"
                   + "\n".join(body) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
    assert mk.SKEWER_DTYPE.itemsize == mk.SKEWER_BYTES


def declared_signatures():
    # {name: [parameter declarations]} of every function in the header
    src = open(os.path.join(ROOT, "include", "mockskewer.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(mk_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        params = [p.strip() for p in m.group(2).split(",")]
        out[m.group(1)] = [] if params == ["void"] else params
    return out


def c_kind(decl):
    # argument class of a C parameter declaration
    if "*" in decl or "[" in decl:
        return "ptr"
    for t, k in (("uint64_t", "u64"), ("int64_t", "i64"), ("uint32_t", "u32"), ("int32_t", "i32"),
                 ("double", "f64"), ("float", "f32"), ("int", "i32")):
        if re.search(rf"\b{t}\b", decl):
            return k
    raise AssertionError(decl)


def ctypes_kind(t):
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return "ptr"
    for ct, k in ((C.c_uint64, "u64"), (C.c_int64, "i64"), (C.c_uint32, "u32"), (C.c_int32, "i32"),
                  (C.c_double, "f64"), (C.c_float, "f32")):
        if C.sizeof(t) == C.sizeof(ct) and t._type_ == ct._type_:
            return k
    raise AssertionError(t)


def test_binding_signatures_match_the_header():
    # every declared function is bound with as many arguments as the header
    # gives it, each of the same class (pointer, integer width, float)
    L = mk.lib()
    sigs = declared_signatures()
    assert sorted(sigs) == declared_symbols()
    for name, params in sigs.items():
        got = [ctypes_kind(t) for t in getattr(L, name).argtypes]
        assert got == [c_kind(p) for p in params], name
    # and the result: int status codes, void, or the error string
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "mockskewer.h")).read(), flags=re.S)
    ret = {m.group(2): m.group(1).strip()
           for m in re.finditer(r"^([A-Za-z_][A-Za-z_0-9 ]*?\s*\**)\s*(mk_[a-z_0-9]+)\s*\(", src, re.M)}
    assert sorted(ret) == sorted(sigs)
    want = {"int": C.c_int, "void": None, "const char *": C.c_char_p}
    for name, r in ret.items():
        assert getattr(L, name).restype is want[r], name
