"""The allocation-free neighbour build, through the C ABI.

pd_build_neighbours_noalloc serves callers that may not allocate device
memory (for example code embedded under an external memory manager that owns
every device allocation): it keeps its one word of scratch in a static device
array instead of calling cudaMalloc. Its output must equal that of
pd_build_neighbours exactly (index work is bit-exact), call after call, since
the static scratch is reused and must be cleared each time. This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import pd_workloads as W

pytestmark = pytest.mark.gpu


def _build(pd, fn, g):
    G = pd.grid_struct(g)
    n = g.nx * g.ny * g.nz
    row = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    nb = ctypes.c_int64(-1)
    rc = fn(ctypes.byref(G), pd._ptr(row), None, 0, ctypes.byref(nb), None)
    assert rc == 0
    col = torch.full((max(nb.value, 1),), -1, dtype=torch.int32, device="cuda")
    rc = fn(ctypes.byref(G), pd._ptr(row), pd._ptr(col), nb.value, ctypes.byref(nb), None)
    assert rc == 0
    torch.cuda.synchronize()
    return row.cpu().numpy(), col[: nb.value].cpu().numpy()


def test_noalloc_matches_allocating_build_twice(built_lib):
    pd = built_lib
    L = pd.lib()
    # two calls in a row (a notched beam, then the bar), each against the allocating entry point
    for g in (W.beam(2.5).grid, W.bar().grid):
        ra, ca = _build(pd, L.pd_build_neighbours, g)
        rb, cb = _build(pd, L.pd_build_neighbours_noalloc, g)
        assert np.array_equal(ra, rb)
        assert np.array_equal(ca, cb)


def test_noalloc_capacity_error_leaves_col_untouched(built_lib):
    pd = built_lib
    L = pd.lib()
    g = W.tiny_beam().grid
    G = pd.grid_struct(g)
    row = torch.empty(g.n_nodes + 1, dtype=torch.int32, device="cuda")
    col = torch.full((10,), -7, dtype=torch.int32, device="cuda")
    nb = ctypes.c_int64(0)
    rc = L.pd_build_neighbours_noalloc(ctypes.byref(G), pd._ptr(row), pd._ptr(col), 10, ctypes.byref(nb), None)
    assert rc == pd.PD_ERR_CAP and nb.value > 10
    assert (col.cpu() == -7).all()


def test_noalloc_overflow_is_reported_and_the_next_call_succeeds(built_lib):
    """A count-only call on a grid of more than 2^31 - 1 bonds (2047 x 2047 x 6
    nodes: 2,477,771,416 directed bonds) sets the overflow flag in the static
    scratch and must fail with PD_ERR_ARG, leaving n_bonds untouched; the next
    call must start from a cleared flag and succeed."""
    pd = built_lib
    L = pd.lib()
    big = W.Grid(2047, 2047, 6, 1e-3, 3.01)
    G = pd.grid_struct(big)
    row = torch.empty(big.n_nodes + 1, dtype=torch.int32, device="cuda")
    nb = ctypes.c_int64(-5)
    rc = L.pd_build_neighbours_noalloc(ctypes.byref(G), pd._ptr(row), None, 0, ctypes.byref(nb), None)
    assert rc == pd.PD_ERR_ARG and nb.value == -5
    buf = ctypes.create_string_buffer(256)
    L.pd_last_error(buf, 256)
    assert b"2^31" in buf.value
    del row
    torch.cuda.empty_cache()
    g = W.bar().grid
    ra, ca = _build(pd, L.pd_build_neighbours, g)
    rb, cb = _build(pd, L.pd_build_neighbours_noalloc, g)
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
