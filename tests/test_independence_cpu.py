"""The oracle and the CUDA path share no code, and the product path has no CPU
fallback (CPU checks; nothing here touches a GPU).

* No module of the package imports the oracle, and the oracle imports nothing
  from the package: the two meet only in the tests, the smoke check and the
  benchmark's CPU legs.
* The CUDA sources include only their own headers, the public header and
  system/CUDA headers; the oracle's C sources include only the C library.
* The only module both sides read is the seeded input generator, and it
  carries none of the solver's arithmetic (no EOS, reconstruction, flux or
  time-stepping routine).
* With the library missing, the binding raises instead of computing anything.
"""
import ast
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2409_10729_gb300")
CSRC = os.path.join(PKG, "csrc")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                names.add(node.module.split(".")[0])
            elif node.level > 0:
                names.add("<relative>")
    # dynamic imports by name
    for m in re.findall(r"import_module\(\s*['\"]([\w.]+)", open(path).read()):
        names.add(m.split(".")[0])
    return names


def _py_files(d):
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_package_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imports(f), f


def test_oracle_never_imports_the_package():
    for f in _py_files(ORACLE):
        imps = _imports(f)
        assert "paper_2409_10729_gb300" not in imps and "<relative>" not in imps, f


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), flags=re.M)


def test_cuda_sources_include_only_their_own_and_system_headers():
    own = set(os.listdir(CSRC)) | {"mfc.h"}
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith((".cu", ".cuh")):
            continue
        for inc in _includes(os.path.join(CSRC, f)):
            assert "oracle" not in inc and "/" not in inc, (f, inc)
            assert inc in own or not inc.endswith((".cuh", ".c")), (f, inc)


def test_oracle_sources_include_only_the_c_library():
    allowed = {"math.h", "stdlib.h", "string.h", "stddef.h", "stdint.h", "float.h"}
    for f in sorted(os.listdir(ORACLE)):
        if f.endswith(".c"):
            assert set(_includes(os.path.join(ORACLE, f))) <= allowed, f


def test_input_generator_carries_none_of_the_solver_arithmetic():
    src = open(os.path.join(PKG, "inputs.py")).read()
    tree = ast.parse(src)
    funcs = {n.name.lower() for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)}
    for word in ("weno", "hllc", "rhs", "flux", "cons", "rk3", "wavespeed", "sound"):
        assert not any(word in fn for fn in funcs), (word, sorted(funcs))
    assert _imports(os.path.join(PKG, "inputs.py")) <= {"__future__", "math", "numpy"}


def test_binding_raises_when_the_library_is_missing(tmp_path):
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2409_10729_gb300 import mfc\n"
        "mfc.LIB_PATH = %r\n"
        "try:\n"
        "    mfc.lib()\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n" % (ROOT, str(tmp_path / "absent" / "libmfc5.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not built" in r.stdout
