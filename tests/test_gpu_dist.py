"""One array spread over G ranks (brev_dist_pack, the exchange,
brev_dist_finish), run on one GPU as G virtual ranks: G device blocks, the
exchange done by plain device copies of the plan's segments.  Every block
must equal its part of the oracle's permutation of the whole array, bit for
bit."""
import numpy as np
import pytest
import torch

from gpu_util import DTYPE, KIND, to_bytes
from paper_1708_01873_gb300 import inputs

pytestmark = pytest.mark.gpu


def _virtual_ranks(brev, oracle, k, g, E, seed):
    G = 1 << g
    n_loc = 1 << (k - g)
    full = inputs.array_np(seed, 1 << k, KIND[E])
    dev = torch.from_numpy(full.copy()).cuda().view(DTYPE[E])
    blocks = [dev[p * n_loc:(p + 1) * n_loc].clone() for p in range(G)]
    recvs = [torch.empty_like(b) for b in blocks]
    sends = [torch.empty_like(b) for b in blocks]
    for p in range(G):                              # step 1 on every rank
        brev.brev_dist_pack(sends[p], blocks[p], k, g)
    for q in range(G):                              # step 2: the exchange
        so, ro, seg = brev.brev_dist_plan(k, g, E, q)
        for p in range(G):
            src_off = brev.brev_dist_plan(k, g, E, p)[0][q]
            recvs[q][ro[p]:ro[p] + seg].copy_(sends[p][src_off:src_off + seg])
    for q in range(G):                              # step 3 on every rank
        brev.brev_dist_finish(blocks[q], recvs[q], k, g)
    torch.cuda.synchronize()
    exp = oracle.brev_oop(full, k, E).reshape(G, -1)
    for p in range(G):
        got = to_bytes(blocks[p])
        assert np.array_equal(got, exp[p]), f"k={k} g={g} E={E}: rank {p} differs"


@pytest.mark.parametrize("E", (16, 8, 4, 2, 1))
def test_virtual_ranks_match_oracle(brev_lib, oracle_lib, cuda_device, E):
    gmax = {16: 5, 8: 5, 4: 6, 2: 7, 1: 8}[E]
    for g in sorted({1, 2, 3, min(gmax, 5)}):
        for k in (2 * g, 2 * g + 1, 2 * g + 5, 17, 22):
            if k < 2 * g:
                continue
            _virtual_ranks(brev_lib, oracle_lib, k, g, E, 300 + 10 * k + g)


def test_pack_in_place_and_one_rank(brev_lib, oracle_lib, cuda_device):
    """The pack may run in place (send = block), and one rank (g = 0) is the
    plain permutation."""
    k, E = 20, 16
    x = inputs.array_np(5, 1 << k, "c128")
    blk = torch.from_numpy(x.copy()).cuda().view(torch.complex128)
    recv = torch.empty_like(blk)
    brev_lib.brev_dist_pack(blk, blk, k, 0)
    recv.copy_(blk)
    brev_lib.brev_dist_finish(blk, recv, k, 0)
    torch.cuda.synchronize()
    assert np.array_equal(to_bytes(blk), oracle_lib.brev_oop(x, k, E))


def test_dist_errors(brev_lib, cuda_device):
    L = brev_lib.lib()
    a = torch.empty(1 << 12, dtype=torch.complex128, device="cuda")
    b = torch.empty_like(a)
    c0 = brev_lib.brev_launch_count()
    assert L.brev_dist_finish(a.data_ptr(), a.data_ptr(), 14, 2, 16, None) == 3  # overlap
    # 2^6 ranks exceed what one finish tile spans for 16-byte elements
    assert L.brev_dist_finish(a.data_ptr(), b.data_ptr(), 18, 6, 16, None) == 6
    assert L.brev_dist_pack(b.data_ptr(), a.data_ptr(), 3, 2, 16, None) == 1     # 2g > k
    assert brev_lib.brev_launch_count() == c0
