"""The quick-start example (examples/quickstart.py) runs as written on the
GPU and does what it says: y (out of place) equals x permuted in place, and
the batched call followed by one plan replay applies the involution twice,
restoring the arrays."""
import os
import runpy

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_quickstart_example(brev_lib, cuda_device):
    torch.manual_seed(0)
    real_randn = torch.randn
    originals = []

    def recording_randn(*args, **kwargs):
        t = real_randn(*args, **kwargs)
        originals.append(t.clone())
        return t

    torch.randn = recording_randn
    try:
        ns = runpy.run_path(os.path.join(ROOT, "examples", "quickstart.py"))
        torch.cuda.synchronize()
    finally:
        torch.randn = real_randn
    assert torch.equal(ns["y"], ns["x"])
    assert not torch.equal(ns["x"], originals[0])
    for a, orig in zip(ns["arrays"], originals[1:]):
        assert torch.equal(a, orig)
    ns["plan"].close()
