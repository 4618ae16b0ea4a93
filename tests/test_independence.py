"""The CUDA path and the oracle share no code and neither imports the other: no module or
source of the package imports, includes or builds anything under oracle/, the oracle neither
imports the package nor includes its headers, and the two callers that may use the oracle
(bench.py's CPU-baseline and reference legs, __graft_entry__'s build and smoke) import it
inside functions only, so the timed product path never loads it. CPU only."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2503_18479_gb300")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_use_the_oracle():
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), path
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", src), path
        assert "liboracle" not in src and "oracle.c" not in src, path
    for path in _files(os.path.join(ROOT, "include"), (".h",)):
        src = open(path).read()
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", src), path
        assert "liboracle" not in src, path


def test_oracle_does_not_use_the_package():
    for path in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        src = open(path).read()
        assert "paper_2503_18479_gb300" not in src, path
        assert not re.search(r"#\s*include\s*[<\"](mts\.h|common\.cuh|kernels\.h)", src), path
        assert "libmts" not in src, path


def test_oracle_imports_of_the_allowed_callers_are_local():
    for name in ("bench.py", "__graft_entry__.py"):
        src = open(os.path.join(ROOT, name)).read()
        for line in src.splitlines():
            if re.match(r"\s*(import|from)\s+oracle\b", line):
                assert line.startswith((" ", "\t")), f"{name}: module-level oracle import: {line!r}"


def test_product_path_fails_loudly_without_the_library(tmp_path):
    """With libmts.so absent the binding raises ImportError at the first call (here: loading
    the library, and building a Simulator), instead of falling back to any CPU code."""
    import subprocess
    import sys
    code = (
        "import sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2503_18479_gb300 import native, workloads as W\n"
        f"native.LIB_PATH = {str(tmp_path / 'absent' / 'libmts.so')!r}\n"
        "for what in ('lib', 'simulator'):\n"
        "    try:\n"
        "        if what == 'lib':\n"
        "            native.lib()\n"
        "        else:\n"
        "            from paper_2503_18479_gb300.simulator import Simulator\n"
        "            Simulator(W.single_loop(seed=0, n_cfg=2, n_freq=2, grid=4), 'mixed', device='cpu')\n"
        "        print(what, 'no error')\n"
        "    except ImportError:\n"
        "        print(what, 'ImportError')\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split("\n")[:2] == ["lib ImportError", "simulator ImportError"], r.stdout
