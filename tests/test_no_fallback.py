"""CPU checks that the product path has no CPU fallback: a missing library
raises on load, a context cannot be made without a GPU, and nothing in the
package imports or names the oracle (which is test infrastructure only)."""
import ast
import os

import pytest
import torch

from paper_2012_11130_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2012_11130_gb300")


def test_missing_library_raises(tmp_path):
    saved = _native._lib
    _native._lib = None
    try:
        with pytest.raises(ImportError, match="missing"):
            _native.load(str(tmp_path / "libsrhd.so"))
    finally:
        _native._lib = saved


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_context_needs_a_gpu():
    from paper_2012_11130_gb300 import srhd
    with pytest.raises(Exception):
        srhd.Context()


def test_package_does_not_import_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for fn in files:
            if not fn.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, fn)).read())
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                for n in names:
                    assert not n.split(".")[0] == "oracle", (fn, n)
                if isinstance(node, ast.Constant) and isinstance(node.value, str):
                    assert "liboracle" not in node.value, fn
