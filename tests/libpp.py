"""Test helper: build (if needed) and load the C-ABI library."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2401_06684_gb300 import build as _build  # noqa: E402
from paper_2401_06684_gb300 import pp  # noqa: E402

_built = False


def load():
    global _built
    if not _built:
        _build.build()
        _built = True
    pp.lib()
    return pp
