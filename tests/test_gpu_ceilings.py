"""The device ceilings the bench divides by, measured by the library:
the FP64 fused multiply-add rate and the SM-driven host-to-host copy rate
over page-locked memory, with their argument checks."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_plausible(brev_lib, cuda_device):
    t = brev_lib.brev_fp64_fma_tflops()
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    # at most 4 FP64 FMA per SM per cycle at 3 GHz: a loose upper bound that
    # catches a kernel whose work was optimised away
    assert 0.05 < t < sm * 4 * 2 * 3.0e9 / 1e12
    assert brev_lib.lib().brev_fp64_fma_tflops(None) == 1


def test_host_link_rate_and_checks(brev_lib, cuda_device):
    L = brev_lib.lib()
    n = 64 << 20
    a = torch.full((n,), 7, dtype=torch.uint8, pin_memory=True)
    b = torch.zeros(n, dtype=torch.uint8, pin_memory=True)
    gbs = brev_lib.brev_host_link_gbs(b, a)
    assert gbs > 1.0
    assert torch.equal(a, b)  # the copy really ran
    v = ctypes.c_double()
    pageable = torch.zeros(n, dtype=torch.uint8)
    assert L.brev_host_link_gbs(pageable.data_ptr(), a.data_ptr(), n, ctypes.byref(v)) == 1
    assert L.brev_host_link_gbs(b.data_ptr(), a.data_ptr(), n - 8, ctypes.byref(v)) == 2
    assert L.brev_host_link_gbs(a.data_ptr() + 16, a.data_ptr(), 1 << 20, ctypes.byref(v)) == 3


def test_workspace_bytes_reports_the_pool(brev_lib, cuda_device):
    x = torch.empty(1 << 16, dtype=torch.complex128, device="cuda")
    brev_lib.brev_permute_batched([x])  # uses stream-ordered workspace
    torch.cuda.synchronize()
    reserved, used = brev_lib.brev_workspace_bytes()
    assert reserved > 0 and used == 0
