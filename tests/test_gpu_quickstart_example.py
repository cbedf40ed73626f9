"""The README's Python example runs as written on the GPU and does what it
says: y (out of place) equals x permuted in place, and the batched call
followed by one plan replay applies the involution twice, restoring the
arrays."""
import os
import re

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example(brev_lib, cuda_device):
    with open(os.path.join(ROOT, "README.md")) as f:
        blocks = re.findall(r"```python\n(.*?)```", f.read(), re.S)
    assert len(blocks) == 1
    torch.manual_seed(0)
    ns = {}
    real_randn = torch.randn
    originals = []

    def recording_randn(*args, **kwargs):
        t = real_randn(*args, **kwargs)
        originals.append(t.clone())
        return t

    torch.randn = recording_randn
    try:
        exec(compile(blocks[0], "README.md", "exec"), ns)
        torch.cuda.synchronize()
    finally:
        torch.randn = real_randn
    assert torch.equal(ns["y"], ns["x"])
    assert not torch.equal(ns["x"], originals[0])
    for a, orig in zip(ns["arrays"], originals[1:]):
        assert torch.equal(a, orig)
    ns["plan"].close()
