"""The product path has no CPU fallback: without the built CUDA library the binding raises instead of
computing anything (checked in a fresh interpreter, so the library this session loaded is not
reused)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = """
import paper_1506_05094_gb300.md as m
m.LIB = "/nonexistent/libmdgb300.so"
m._lib = None
try:
    m.Sim([100], [10.0], [[1.0]], [[1.0]], [[2.5]])
except ImportError as e:
    print("RAISED:", e)
"""


def test_binding_raises_without_the_cuda_library():
    out = subprocess.run([sys.executable, "-c", CODE], cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert "RAISED:" in out.stdout, (out.stdout, out.stderr)
    assert "has not been built" in out.stdout
