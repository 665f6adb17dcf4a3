"""CPU test: libgp.so and the oracle build, load, and export every symbol
that include/gp.h declares (no compute call: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1203_1269_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_paper_calls():
    names = declared_symbols()
    for n in ("gp_corr_assemble", "gp_nll_batch", "gp_fit", "gp_predict"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_without_gpu_fails_cleanly(lib):
    # no CUDA device in this container: gp_create must return an error code
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.gp_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t,
                              ctypes.c_void_p]
    rc = lib.gp_create(ctypes.byref(h), 0, 0, None)
    assert rc != 0 and not h.value


def test_oracle_builds_and_loads():
    import oracle
    assert oracle.num_threads() >= 1


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU or PyTorch fallback: with libgp.so absent the binding raises,
    for the sizing query as for the compute calls."""
    from paper_1203_1269_gb300 import gp
    monkeypatch.setattr(gp, "_lib", None)
    monkeypatch.setattr(gp._build, "LIB", str(tmp_path / "libgp.so"))
    with pytest.raises(RuntimeError, match="libgp.so not found"):
        gp.load()
    with pytest.raises(RuntimeError, match="libgp.so not found"):
        gp.call_bytes("fit", 100, 2)
    with pytest.raises(RuntimeError, match="libgp.so not found"):
        gp.Context(0)


def _declared_params():
    """Parameter count of every gp_* function gp.h declares."""
    out = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(gp_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every function the Python binding calls has argtypes of the length
    gp.h declares (a drifted signature would pass arguments in the wrong
    registers)."""
    from paper_1203_1269_gb300 import gp
    lib = gp.load()
    declared = _declared_params()
    bound = {name: len(getattr(lib, name).argtypes) for name in declared
             if getattr(getattr(lib, name), "argtypes", None) is not None}
    assert len(bound) >= 25, sorted(bound)
    wrong = {k: (v, declared[k]) for k, v in bound.items() if v != declared[k]}
    assert not wrong, wrong
    # and the binding sets argtypes for every call it makes
    src = open(os.path.join(ROOT, "paper_1203_1269_gb300", "gp.py")).read()
    called = set(re.findall(r"_lib\.(gp_[a-z0-9_]+)\(", src)) | set(re.findall(r"\blib\.(gp_[a-z0-9_]+)\(", src))
    assert called <= set(bound), sorted(called - set(bound))


def _declared_struct(name):
    """(field, C type) pairs of the typedef struct `name` in gp.h, in order."""
    src = open(os.path.join(ROOT, "include", "gp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + name + r"\s*;", src, flags=re.S)
    assert m, name
    return re.findall(r"\b(int|double)\s+([a-z_0-9]+)\s*;", m.group(1))


@pytest.mark.parametrize("cname,pyname", [("gp_options", "Options"), ("gp_tune_trial", "TuneTrial")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes structures the binding passes by pointer have gp.h's
    fields, in its order and with its types."""
    import ctypes
    from paper_1203_1269_gb300 import gp
    want = [(f, {"int": ctypes.c_int, "double": ctypes.c_double}[t]) for t, f in _declared_struct(cname)]
    assert len(want) >= 4
    assert list(getattr(gp, pyname)._fields_) == want


def test_oracle_wrapper_signatures_match_the_source():
    """The oracle's ctypes wrapper passes as many arguments as each exported
    gpo_* function of gp_oracle.c takes, in both of its builds."""
    import oracle
    src = open(os.path.join(ROOT, "oracle", "gp_oracle.c")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    declared = {}
    for m in re.finditer(r"^(?!static)[a-z][a-z ]*\b(gpo_[a-z0-9_]+)\s*\(([^)]*)\)\s*\{", src, flags=re.M):
        params = m.group(2).strip()
        declared[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    assert len(declared) >= 10, declared
    for orc in (oracle.default(), oracle.extended()):
        for name, count in declared.items():
            assert len(getattr(orc.lib, name).argtypes or ()) == count, name
