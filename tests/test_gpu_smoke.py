"""The smoke entry point (`__graft_entry__.smoke()`): its three cases pass on
the GPU with the library as built."""
import os
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")


def test_smoke_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.smoke()
