"""The FP64 band panels' overlaps on the library's side streams (each panel's
U12 beside its L21; the look-ahead of the trailing update) against the serial
order and the CPU oracle.

Every entry receives the same operations in the same order in every mode,
so the factors must agree bit for bit; against the oracle's banded
Doolittle within 1e-13.  The factorisation is also captured into a CUDA
graph (the side streams fork from and join the capturing stream) and
replayed.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture
def overlap_mode():
    lib = ebv.lib()
    yield lambda m: lib.ebv_debug_set_band_lookahead(m)
    lib.ebv_debug_set_band_lookahead(2)


def _band(n, kl, ku, seed):
    a = synthetic.dense_dd(n, 0.9, seed)
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[(d > kl) | (d < -ku)] = 0.0
    return synthetic.dense_to_band(a, kl, ku)


@pytest.mark.parametrize("n,kl,ku", [(700, 130, 200), (1000, 64, 64), (513, 5, 300), (300, 250, 3)])
def test_modes_bitwise_equal(overlap_mode, n, kl, ku):
    ab = _band(n, kl, ku, 95_000 + n)
    fb, _ = oracle.band_lu(ab, kl, ku)
    out = {}
    for mode in (0, 1, 2):
        overlap_mode(mode)
        f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, "fp64")
        assert int(f.info.item()) == 0
        out[mode] = f.lu.cpu().numpy()
        assert np.abs(out[mode] - fb).max() <= 1e-13, mode
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("mode", [1, 2])
def test_graph_capture_with_side_streams(overlap_mode, mode):
    n, kl, ku = 900, 100, 150
    ab = _band(n, kl, ku, 96_000)
    overlap_mode(mode)
    AB = torch.from_numpy(ab).to(DEV)
    lu = AB.clone()
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = ebv.workspace(n, "fp64", 1, DEV, kl=kl, ku=ku, storage=ebv.BAND)
    ebv.ebv_factor(lu, "fp64", info=info, ws=ws, kl=kl, ku=ku, storage=ebv.BAND)  # creates the side streams
    torch.cuda.synchronize()
    ref = lu.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lu.copy_(AB)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws, kl=kl, ku=ku, storage=ebv.BAND)
    lu.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert torch.equal(lu, ref)
