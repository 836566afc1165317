"""Test helpers: build and import the CUDA library (no oracle code here)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def dlz():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "dlz_build", os.path.join(ROOT, "paper_0901_3163_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    from paper_0901_3163_gb300 import dlz as mod
    return mod
