"""The product path never uses the oracle: no module of the package and no
CUDA source imports, includes or loads anything under oracle/, and the
package's loader fails loudly (no CPU fallback) when the library is absent."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_20374_gb300")


def _sources():
    for base, _, files in os.walk(PKG):
        if "_build" in base or "__pycache__" in base:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                yield os.path.join(base, f)


def test_package_sources_do_not_reference_the_oracle():
    bad = []
    for path in _sources():
        text = open(path).read()
        if re.search(r"^\s*(import|from)\s+oracle\b", text, re.M) or "ncorp_oracle" in text or "oracle/" in text:
            bad.append(os.path.relpath(path, ROOT))
    assert not bad, bad


def test_oracle_and_product_share_no_source():
    oracle_dir = os.path.join(ROOT, "oracle")
    oracle_text = "".join(open(os.path.join(oracle_dir, f)).read()
                          for f in os.listdir(oracle_dir) if f.endswith((".c", ".py")))
    assert "paper_2310_20374_gb300" not in oracle_text
    assert "#include \"" not in open(os.path.join(oracle_dir, "ncorp_oracle.c")).read()


def test_loader_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2310_20374_gb300 import build as B
    from paper_2310_20374_gb300 import ncorp
    monkeypatch.setattr(ncorp, "_lib", None)
    monkeypatch.setattr(B, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        ncorp.load()
