"""The oracle and the CUDA path share no code, and only the test
infrastructure runs the oracle: a static scan of the committed sources.

* Nothing in the package (Python, C++, CUDA) imports, includes, links or
  loads anything from ``oracle/``.
* Nothing in ``oracle/`` refers to the package, its header or its library.
* The seeded input generators (``synthetic/``) import neither side.
* Outside ``tests/``, only ``__graft_entry__.py`` (its build and smoke check) and
  ``bench.py`` (its CPU baseline and oracle arm, inside those functions only)
  import the oracle.
* The oracle's C sources include nothing but the C standard library."""
import ast
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1908_07038_gb300"


def _ignored_dirs():
    """Directory names the repository's .gitignore lists (plain names and
    paths, not patterns), plus .git: what a copy without git history skips."""
    names = {".git"}
    try:
        with open(os.path.join(ROOT, ".gitignore"), encoding="utf-8") as fh:
            for line in fh:
                line = line.strip()
                if line and not line.startswith("#") and not any(c in line for c in "*?["):
                    names.add(line.strip("/").split("/")[0])
    except OSError:
        pass
    return names


SKIP_DIRS = _ignored_dirs()


def _files(prefix, exts):
    """Committed files under prefix (git), or, in a copy without its git
    history, the source files found there."""
    try:
        out = subprocess.check_output(["git", "ls-files", prefix], cwd=ROOT, text=True,
                                      stderr=subprocess.DEVNULL).split()
    except (OSError, subprocess.CalledProcessError):
        out = []
        for d, dirs, names in os.walk(os.path.join(ROOT, prefix)):
            dirs[:] = [x for x in dirs if x not in SKIP_DIRS]
            out += [os.path.relpath(os.path.join(d, n), ROOT) for n in names]
    return sorted(f for f in out if f.endswith(exts))


def _text(path):
    with open(os.path.join(ROOT, path), encoding="utf-8") as fh:
        return fh.read()


def _imports(path):
    """(module names imported, (function or None) they are imported in)."""
    tree = ast.parse(_text(path))
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                found.extend((a.name, func) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module:
                found.append((child.module, func))
            visit(child, f)

    visit(tree, None)
    return found


def test_package_never_reaches_the_oracle():
    for f in _files(PKG, (".py",)):
        for mod, _ in _imports(f):
            assert not (mod == "oracle" or mod.startswith("oracle.")), (f, mod)
    for f in _files(PKG, (".py", ".cpp", ".cu", ".h")):
        t = _text(f)
        assert not re.search(r"#include\s+[\"<][^\">]*oracle", t), f
        assert "liboracle" not in t and "orc_" not in t, f


def _c_code(text):
    """C source without its comments (the oracle's header may name the
    package to say that it never links it)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def test_oracle_never_reaches_the_package():
    for f in _files("oracle", (".c", ".h")):
        t = _c_code(_text(f))
        for word in (PKG, "atlas_gb.h", "libatlasgb", "csrc"):
            assert word not in t, (f, word)
    for f in _files("oracle", (".py",)):
        for mod, _ in _imports(f):
            assert not mod.startswith(PKG), (f, mod)
        # no path or name of the product in any string the code uses
        tree = ast.parse(_text(f))
        docs = {id(n.body[0].value) for n in ast.walk(tree)
                if isinstance(n, (ast.Module, ast.FunctionDef, ast.ClassDef)) and n.body
                and isinstance(n.body[0], ast.Expr) and isinstance(n.body[0].value, ast.Constant)}
        for n in ast.walk(tree):
            if isinstance(n, ast.Constant) and isinstance(n.value, str) and id(n) not in docs:
                for word in (PKG, "libatlasgb", "atlas_gb"):
                    assert word not in n.value, (f, n.value)


def test_input_generators_import_neither_side():
    for f in _files("synthetic", (".py",)):
        for mod, _ in _imports(f):
            top = mod.split(".")[0]
            assert top not in ("oracle", PKG), (f, mod)


def test_only_test_infrastructure_imports_the_oracle():
    # build() compiles the oracle's C library (building the checker is not
    # running it); smoke() checks one small GPU call against it
    allowed = {"__graft_entry__.py": {"build", "smoke"}, "bench.py": {"_cpu_baseline", "run_reference"}}
    for f in _files(".", (".py",)):
        if f.startswith(("tests/", "oracle/")):
            continue
        for mod, func in _imports(f):
            if mod == "oracle" or mod.startswith("oracle."):
                assert f in allowed and func in allowed[f], (f, mod, func)


def test_oracle_c_sources_include_only_the_standard_library():
    std = {"math.h", "stdint.h", "stdlib.h", "string.h", "stdio.h", "stddef.h", "float.h"}
    for f in _files("oracle", (".c", ".h")):
        for inc in re.findall(r"#include\s+[\"<]([^\">]+)[\">]", _text(f)):
            assert inc in std, (f, inc)
