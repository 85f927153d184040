"""The allocation-free counting sort (aica_sort_by_cell_noalloc).

Some callers cannot allocate device memory while they run: work recorded
into a CUDA graph or stream capture, real-time loops, hosts whose device
memory belongs to another allocator.  For them the library offers a sort by
cell whose workspace is a fixed device array inside the library.  These tests
check, through the C ABI, that it reproduces the binned order and cell
offsets of aica_bin_molecules exactly (integers), on two calls in a row that
reuse the shared workspace, and that it rejects more cells than its
workspace holds.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_cs_0702131_gb300 import aica, synth


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
    L = aica.lib()
    for call in range(2):
        o2 = torch.full_like(order, -7)
        off2 = torch.full_like(cell_off, -7)
        st = L.aica_sort_by_cell_noalloc(ctypes.c_void_p(cell_of.data_ptr()), cell_of.numel(), C,
                                         ctypes.c_void_p(o2.data_ptr()), ctypes.c_void_p(off2.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, L.aica_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o2.cpu().numpy(), order.cpu().numpy(), err_msg=f"call {call}")
        np.testing.assert_array_equal(off2.cpu().numpy(), cell_off.cpu().numpy(), err_msg=f"call {call}")
    m.close()
