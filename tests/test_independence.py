"""The rules that keep the parity claims honest, checked on the source and on the host:
the package (the product path) never imports the oracle or the CPU baseline; the oracle and the
CPU baseline include nothing from the CUDA library; and the product path fails loudly when its
CUDA library is missing instead of falling back to anything else."""
import ast
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1303_1651_gb300")


def imported_modules(path):
    tree = ast.parse(open(path).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name.split(".")[0]
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            yield node.module.split(".")[0]


def test_package_never_imports_the_oracle_or_baseline():
    files = glob.glob(os.path.join(PKG, "*.py"))
    assert files
    for f in files:
        bad = {m for m in imported_modules(f)} & {"oracle", "baseline", "tests", "bench"}
        assert not bad, f"{os.path.basename(f)} imports {bad}"
    for f in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(f).read()
        assert "oracle" not in re.findall(r'#include\s+"([^"]+)"', text), f


def test_oracle_and_baseline_share_nothing_with_the_cuda_library():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "baseline", "*.cpp")):
        includes = re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(f).read())
        for inc in includes:
            assert not os.path.exists(os.path.join(PKG, "csrc", inc)), f"{f} includes {inc} of the CUDA library"
            assert not inc.startswith("cuda") and "spgemm_gb300" not in inc, f"{f} includes {inc}"
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")) + glob.glob(os.path.join(ROOT, "baseline", "*.py")):
        assert "paper_1303_1651_gb300" not in set(imported_modules(f)), f


def test_product_path_fails_loudly_without_its_library(monkeypatch, tmp_path):
    from paper_1303_1651_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()
