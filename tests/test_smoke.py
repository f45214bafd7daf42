"""The package entry point's smoke() (one small energy + exact-gradient evaluation on cuda:0,
checked against the oracle) runs and passes."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    torch = pytest.importorskip("torch")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import __graft_entry__ as entry
    entry.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.smoke()
