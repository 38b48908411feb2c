"""The smoke entry point (marked gpu): both of its legs, the one-orbital FP64 run and
the 64-orbital split-FP16 run in the benchmark's kernel configuration, match the
oracle."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import torch

    import __graft_entry__ as g
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    g.smoke()
