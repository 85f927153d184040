"""The allocation-free counting sort (aica_sort_by_cell_noalloc).

Some callers cannot allocate device memory while they run: work recorded
into a CUDA graph or stream capture, real-time loops, hosts whose device
memory belongs to another allocator.  For them the library offers a sort by
cell whose workspace is a fixed device array inside the library.  These tests
check, through the C ABI, that it reproduces the binned order and cell
offsets of aica_bin_molecules and of the oracle's stable counting sort
exactly (integers), on two calls in a row that reuse the shared workspace;
that a cell id beyond n_cells is left out like -1 without any access outside
the arrays; and that it rejects more cells than its workspace holds.  This
file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_cs_0702131_gb300 import aica, synth


def _sort(L, cell_of, C, order, cell_off):
    return L.aica_sort_by_cell_noalloc(ctypes.c_void_p(cell_of.data_ptr()), cell_of.numel(), C,
                                       ctypes.c_void_p(order.data_ptr()), ctypes.c_void_p(cell_off.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_rejects_more_cells_than_the_workspace():
    L = aica.lib()
    st = L.aica_sort_by_cell_noalloc(None, 0, (1 << 20) + 1, None, ctypes.c_void_p(8), None)
    assert aica.STATUS[st] == "AICA_ERR_CAPACITY"
    assert b"workspace" in L.aica_last_error()


@pytest.mark.gpu
def test_noalloc_sort_equals_binning_twice():
    c = synth.make("c2", 5)
    m = aica.Mesh(c["mesh"], c["box"])
    m.build_lists(c["rc"], c["skin"])
    pos = torch.tensor(c["pos"], dtype=torch.float64, device="cuda")
    sp = torch.tensor(c["species"], dtype=torch.int32, device="cuda")
    cell_of, order, cell_off = m.bin(pos, sp)
    C = c["mesh"]["n_cells"]
    o_order, o_off = oracle.bin_order(cell_of.cpu().numpy(), C)
    L = aica.lib()
    for call in range(2):
        o2 = torch.full_like(order, -7)
        off2 = torch.full_like(cell_off, -7)
        st = _sort(L, cell_of, C, o2, off2)
        assert st == 0, L.aica_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o2.cpu().numpy(), order.cpu().numpy(), err_msg=f"call {call}")
        np.testing.assert_array_equal(off2.cpu().numpy(), cell_off.cpu().numpy(), err_msg=f"call {call}")
        np.testing.assert_array_equal(o2.cpu().numpy(), o_order, err_msg=f"oracle, call {call}")
        np.testing.assert_array_equal(off2.cpu().numpy(), o_off, err_msg=f"oracle, call {call}")
    m.close()


@pytest.mark.gpu
def test_noalloc_sort_leaves_out_ids_beyond_n_cells():
    rng = np.random.default_rng(3)
    C, n = 5000, 40000
    cells = rng.integers(0, C, n).astype(np.int32)
    cells[rng.choice(n, 50, replace=False)] = -1
    cells[:64] = 7                                   # one crowded cell (bitonic path)
    bad = rng.choice(np.arange(64, n), 3, replace=False)
    cells[bad] = [C, C + 5, 1 << 30]                 # out of range: treated like -1
    expect = cells.copy()
    expect[bad] = -1
    valid = np.flatnonzero(expect >= 0)
    sub, o_off = oracle.bin_order(expect[valid], C)
    o_order = valid[sub]
    L = aica.lib()
    d_cells = torch.tensor(cells, device="cuda")
    pad = 1024                                       # guard region after the arrays
    order = torch.full((n + pad,), -7, dtype=torch.int32, device="cuda")
    off = torch.full((C + 1 + pad,), -7, dtype=torch.int32, device="cuda")
    for call in range(2):
        st = _sort(L, d_cells, C, order, off)
        assert st == 0, L.aica_last_error()
        torch.cuda.synchronize()
        got_off = off.cpu().numpy()
        got = order.cpu().numpy()
        np.testing.assert_array_equal(got_off[:C + 1], o_off)
        placed = int(o_off[-1])
        assert placed == int((expect >= 0).sum()) == int((cells >= 0).sum()) - 3
        np.testing.assert_array_equal(got[:placed], o_order)
        assert (got_off[C + 1:] == -7).all() and (got[n:] == -7).all(), "write outside the arrays"
