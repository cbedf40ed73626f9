"""Helpers shared by the GPU tests: seeded device/host inputs and byte
comparison.  Inputs come from the seeded generator; expected values come from
the CPU oracle only."""
import numpy as np
import torch

from paper_1708_01873_gb300 import inputs

KIND = {1: "u8", 2: "u16", 4: "f32", 8: "c64", 16: "c128"}
DTYPE = {1: torch.uint8, 2: torch.int16, 4: torch.float32, 8: torch.complex64,
         16: torch.complex128}


def device_array(seed: int, k: int, E: int, kind: str | None = None,
                 extra_elems: int = 0) -> torch.Tensor:
    """2^k (+extra) seeded elements on cuda:0, as a tensor of element size E."""
    n = (1 << k) + extra_elems
    raw = torch.empty(n * E, dtype=torch.uint8, device="cuda")
    inputs.fill_torch(raw, seed, kind or KIND[E])
    return raw.view(DTYPE[E])


def host_array(seed: int, k: int, E: int, kind: str | None = None) -> np.ndarray:
    return inputs.array_np(seed, 1 << k, kind or KIND[E])


def to_bytes(t: torch.Tensor) -> np.ndarray:
    return t.detach().contiguous().view(torch.uint8).cpu().numpy().reshape(-1)


def assert_bytes_equal(got: np.ndarray, exp: np.ndarray, E: int, what: str = "") -> None:
    if got.size == exp.size and np.array_equal(got, exp):
        return
    g = got.reshape(-1, E)
    e = exp.reshape(-1, E)
    bad = np.nonzero((g != e).any(axis=1))[0]
    raise AssertionError(f"{what}: {bad.size} of {e.shape[0]} elements differ; "
                         f"first at {bad[:8].tolist()}")
