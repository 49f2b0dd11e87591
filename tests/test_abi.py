"""The C ABI library loads and exports every entry point that include/vc.h declares, a missing
library is an error rather than a fallback, and the package never loads the oracle (no GPU)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:int|const char\s*\*|void)\s*\*?\s*(vc_\w+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_10402_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_symbols()
    for want in ("vc_mvc", "vc_pvc", "vc_mvc_batch"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_names_match_header():
    import paper_2204_10402_gb300 as vc
    assert set(declared_symbols()) == set(vc.EXPORTED)


def test_host_only_calls(lib):
    lib.vc_version.restype = ctypes.c_int
    assert lib.vc_version() >= 100
    lib.vc_strerror.restype = ctypes.c_char_p
    assert lib.vc_strerror(-1) == b"VC_EINVAL"
    assert lib.vc_strerror(0) == b"VC_OK"


def _c_layout(tmp_path, type_name, fields, header):
    """sizeof and field offsets of a C struct, from a tiny C program compiled with the host gcc."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = [f'#include "{header}"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {",
             f'  printf("%zu\\n", sizeof({type_name}));']
    lines += [f'  printf("%zu\\n", offsetof({type_name}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src = tmp_path / f"{type_name}.c"
    exe = tmp_path / f"{type_name}.out"
    src.write_text("\n".join(lines))
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("type_name,header,cls", [
    ("vc_graph", "vc.h", "Graph"), ("vc_config", "vc.h", "Config"), ("vc_stats", "vc.h", "Stats"),
    ("vc_request_info", "vc_server.h", "RequestInfo"), ("vc_server_counters", "vc_server.h", "ServerCounters")])
def test_struct_layouts_match_binding(tmp_path, type_name, header, cls):
    # The ctypes mirrors must have the C structs' sizes and field offsets exactly.
    import paper_2204_10402_gb300 as vc
    py = getattr(vc, cls)
    fields = [name for name, _ in py._fields_]
    size, offsets = _c_layout(tmp_path, type_name, fields, header)
    assert ctypes.sizeof(py) == size
    assert [getattr(py, f).offset for f in fields] == offsets


def test_missing_library_fails_loudly(tmp_path):
    # No CPU fallback: a solve without libvc.so raises instead of computing anything.
    missing = str(tmp_path / "libvc.so")
    code = ("import paper_2204_10402_gb300 as vc\n"
            "from paper_2204_10402_gb300 import graphs as G\n"
            f"vc.LIB_PATH = {missing!r}\n"
            "g = G.path(3)\n"
            "try:\n"
            "    vc.mvc(g.offsets, g.neighbors)\n"
            "except ImportError:\n"
            "    print('raised')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "raised"


def test_product_path_does_not_touch_the_oracle():
    # The oracle is test infrastructure: importing the package and its modules never loads it,
    # and no module of the package names it in an import.
    code = ("import sys\n"
            "import paper_2204_10402_gb300\n"
            "from paper_2204_10402_gb300 import graphs, autotune, build\n"
            "print('oracle' in sys.modules)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "False"
    pkg = os.path.join(ROOT, "paper_2204_10402_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            text = open(os.path.join(pkg, name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name


def test_host_csr_arrays_are_checked_not_wrapped():
    # Host CSR arrays become int32 copies; values outside int32 and non-integer arrays are errors
    # instead of silently wrapped or truncated inputs.
    import numpy as np
    sys.path.insert(0, ROOT)
    import paper_2204_10402_gb300 as vc
    ok = vc._host_i32(np.array([0, 2, 4], dtype=np.int64))
    assert ok.dtype == np.int32 and ok.tolist() == [0, 2, 4]
    assert vc._host_i32([]).size == 0
    with pytest.raises(ValueError):
        vc._host_i32(np.array([0, 2**31], dtype=np.int64))
    with pytest.raises(ValueError):
        vc._host_i32(np.array([-2**31 - 1, 0], dtype=np.int64))
    with pytest.raises(TypeError):
        vc._host_i32(np.array([0.0, 1.5]))
