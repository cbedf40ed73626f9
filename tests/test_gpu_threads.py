"""Several host threads drive the library at once, each on its own stream
(single, batched, plan and host-path calls interleaved): every result equals
the CPU oracle and error messages stay per thread."""
import threading

import numpy as np
import pytest
import torch

from gpu_util import DTYPE, assert_bytes_equal, device_array, host_array, to_bytes

pytestmark = pytest.mark.gpu


def test_concurrent_host_threads(brev_lib, oracle_lib, cuda_device):
    errors = []
    results = {}

    def worker(tid):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            rng = np.random.default_rng(tid)
            for it in range(12):
                k = int(rng.integers(8, 20))
                E = int(rng.choice([4, 8, 16]))
                seed = 100000 + 1000 * tid + it
                with torch.cuda.stream(s):
                    a = device_array(seed, k, E)
                    mode = it % 4
                    if mode == 0:
                        out = torch.empty_like(a)
                        brev_lib.brev_permute_to(out, a, stream=s)
                    elif mode == 1:
                        brev_lib.brev_permute(a, in_place=True, stream=s)
                        out = a
                    elif mode == 2:
                        brev_lib.brev_permute_batched([a], stream=s)
                        out = a
                    else:
                        plan = brev_lib.BrevPlan([a])
                        plan.launch(s)
                        out = a
                    # a failing call on this thread must not leak its message
                    with pytest.raises(brev_lib.BrevError):
                        brev_lib.brev_permute_shape(a, a, 3, 4)
                s.synchronize()
                results[(tid, it)] = (k, E, seed, to_bytes(out))
                if mode == 3:
                    plan.close()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append((tid, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not errors, errors
    assert len(results) == 6 * 12
    for (tid, it), (k, E, seed, got) in results.items():
        exp = oracle_lib.brev_oop(host_array(seed, k, E), k, E)
        assert_bytes_equal(got, exp, E, f"thread {tid} call {it}")
