"""The oracle and the CUDA path are independent, and only test
infrastructure runs the oracle: nothing in the package (Python, CUDA, C)
names the oracle; the oracle's C source includes only standard headers and
its Python wrapper imports nothing from the package; the two shared
libraries export disjoint symbol sets; and in bench.py and
__graft_entry__.py the oracle is imported only inside the CPU-baseline
sampler, build() and smoke(). The seeded input generators are the one module
both sides use, and it imports neither of them; the scripts that write the
stored goldens use only the oracle and those generators. CPU only."""
import ast
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1802_03760_b300")
SOURCE_EXT = (".py", ".cu", ".cuh", ".c", ".h", ".cpp")


def _sources(top):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build")]
        for f in files:
            if f.endswith(SOURCE_EXT):
                yield os.path.join(d, f)


def _code_without_comments(path):
    text = open(path).read()
    if path.endswith(".py"):
        # drop docstrings and comments: only code may not name the oracle
        tree = ast.parse(text)
        names = set()
        for node in ast.walk(tree):
            if isinstance(node, ast.Name):
                names.add(node.id)
            elif isinstance(node, ast.Attribute):
                names.add(node.attr)
            elif isinstance(node, (ast.Import, ast.ImportFrom)):
                for a in node.names:
                    names.add(a.name)
                if isinstance(node, ast.ImportFrom) and node.module:
                    names.add(node.module)
            elif isinstance(node, ast.Constant) and isinstance(node.value, str) and node.value.endswith(".so"):
                names.add(node.value)
        return " ".join(sorted(names))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_package_never_names_the_oracle():
    for path in _sources(PKG):
        code = _code_without_comments(path)
        for word in ("oracle", "gj_oracle", "libgjoracle", "og_count", "og_graph"):
            assert word not in code, (os.path.relpath(path, ROOT), word)


def test_oracle_uses_nothing_from_the_package():
    src = open(os.path.join(ROOT, "oracle", "gj_oracle.c")).read()
    includes = re.findall(r"#\s*include\s*([<\"][^>\"]+[>\"])", src)
    assert includes and all(i.startswith("<") for i in includes), includes
    assert set(includes) <= {"<stdint.h>", "<stdlib.h>", "<string.h>"}, includes
    tree = ast.parse(open(os.path.join(ROOT, "oracle", "__init__.py")).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            assert all(not a.name.startswith("paper_1802_03760_b300") for a in node.names)
        if isinstance(node, ast.ImportFrom):
            assert not (node.module or "").startswith("paper_1802_03760_b300")


def test_input_generators_import_neither_side():
    tree = ast.parse(open(os.path.join(PKG, "inputs", "__init__.py")).read())
    for node in ast.walk(tree):
        mods = [a.name for a in node.names] if isinstance(node, ast.Import) else \
            [node.module or ""] if isinstance(node, ast.ImportFrom) else []
        for m in mods:
            assert not m.startswith("oracle") and "gj" not in m.split("."), m
    gen = open(os.path.join(PKG, "inputs", "gen.c")).read()
    assert set(re.findall(r"#\s*include\s*([<\"][^>\"]+[>\"])", gen)) <= {"<stdint.h>", "<stdlib.h>", "<string.h>"}


def _oracle_imports(path):
    """(line, enclosing function names) of every import of the oracle package."""
    out = []

    def walk(node, stack):
        for ch in ast.iter_child_nodes(node):
            s = stack + [ch.name] if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else stack
            if isinstance(ch, ast.Import):
                mods = [a.name for a in ch.names]
            elif isinstance(ch, ast.ImportFrom):
                mods = [ch.module or ""]
            else:
                mods = []
            if any(m.split(".")[0] == "oracle" for m in mods):
                out.append((ch.lineno, s))
            walk(ch, s)

    walk(ast.parse(open(path).read()), [])
    return out


def test_oracle_runs_only_in_the_baseline_build_and_smoke():
    bench = _oracle_imports(os.path.join(ROOT, "bench.py"))
    assert bench and all(stack and stack[-1] == "cpu_sample" for _, stack in bench), bench
    entry = _oracle_imports(os.path.join(ROOT, "__graft_entry__.py"))
    assert entry and all(stack and stack[0] in ("build", "smoke") for _, stack in entry), entry


def test_libraries_export_disjoint_symbols():
    if shutil.which("nm") is None:
        pytest.skip("nm is not installed")
    from paper_1802_03760_b300.build import build
    import oracle

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
        return {line.split()[-1] for line in out.splitlines() if line.strip()}

    lib, ora = exported(build()), exported(oracle.build())
    assert not any(s.startswith("og_") for s in lib)
    assert not any(s.startswith("gj_") for s in ora)
    assert {"og_count_ex", "og_delta_each"} <= ora and {"gj_count_many", "gj_apply_batch"} <= lib


def test_golden_writers_call_only_the_oracle():
    """Every stored expected value is written by a script that uses the
    oracle and the input generators only: no CUDA binding, no torch."""
    gdir = os.path.join(ROOT, "tests", "golden")
    scripts = sorted(f for f in os.listdir(gdir) if f.endswith(".py"))
    assert scripts
    for f in scripts:
        tree = ast.parse(open(os.path.join(gdir, f)).read())
        mods = set()
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods |= {a.name for a in node.names}
            elif isinstance(node, ast.ImportFrom):
                mods.add(node.module or "")
        pkg = {m for m in mods if m.startswith("paper_1802_03760_b300")}
        assert pkg <= {"paper_1802_03760_b300.inputs"}, (f, pkg)
        assert "oracle" in mods and not any(m.split(".")[0] == "torch" for m in mods), (f, mods)
