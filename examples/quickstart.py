"""Quick start: one array out of place and in place, then a batch of arrays
in one persistent launch and as a captured plan (needs a CUDA GPU and the
built library)."""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1708_01873_gb300 import brev

x = torch.randn(1 << 24, dtype=torch.complex64, device="cuda")
y = torch.empty_like(x)
brev.brev_permute_to(y, x)               # y[rev(i)] = x[i]
brev.brev_permute(x, in_place=True)      # in place (tile pairs swapped)

arrays = [torch.randn(1 << k, dtype=torch.complex128, device="cuda") for k in (8, 12, 20)]
brev.brev_permute_batched(arrays)        # one persistent launch for all of them
plan = brev.BrevPlan(arrays)             # or capture once and replay
plan.launch()
