"""Shared helpers for the tests: build the library on demand and marshal inputs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def ensure_built():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_tn_build", os.path.join(ROOT, "paper_2606_01852_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2606_01852_gb300 as tn
    return tn
