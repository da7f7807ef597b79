"""The allocation-free colouring entry point (amg_colour_noalloc).

Callers that may not allocate at call time (stream capture, real-time paths,
pre-reserved memory) get the finest-level colouring from a fixed device array
inside the library.  This checks, through the C ABI, that it gives exactly the
colouring that amg_setup computes for level 0 (colourings are compared bit for
bit, as everywhere in these tests), on two calls in a row that share the
scratch array; that a setup on a smaller graph between two calls does not
break the next call; that a call captured into a CUDA graph replays to the
same colouring and that warm calls take no device memory; and that patterns
which break the stored-pattern conventions (a block stored on one side only)
are reported with n_colours = -1.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_07537_gb300 import bamg, problems as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _level0_colours(s):
    rp = torch.from_numpy(s.row_ptr).cuda()
    ci = torch.from_numpy(s.col_idx).cuda()
    va = torch.from_numpy(np.ascontiguousarray(s.vals.reshape(-1))).cuda()
    g = bamg.Solver(rp, ci, va, s.b, s.field_of_dof, max_levels=2, max_coarse=0)
    L0 = g.level(0)
    return rp, ci, L0["colour"], L0["n_colours"]


def _call(lib, rp, ci, n, colour, nc, stream):
    return lib.amg_colour_noalloc(rp.data_ptr(), ci.data_ptr(), n, colour.data_ptr(), nc.data_ptr(),
                                  ctypes.c_void_p(stream))


def _outputs(n):
    return (torch.full((n,), -7, dtype=torch.int32, device="cuda"),
            torch.full((1,), -7, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("system", ["mhd2d_40", "stokes3d_9"])
def test_noalloc_colouring_equals_setup_colouring_on_two_calls(system):
    assert torch.cuda.is_available()
    s = P.mhd2d(40, 2) if system == "mhd2d_40" else P.stokes3d(9, 1)
    rp, ci, ref_colour, ref_nc = _level0_colours(s)
    lib = bamg.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        colour, nc = _outputs(s.n_nodes)
        st = _call(lib, rp, ci, s.n_nodes, colour, nc, stream)
        assert st == bamg.BAMG_OK, (call, bamg.amg_strerror(st))
        torch.cuda.synchronize()
        assert int(nc.item()) == ref_nc, call
        assert np.array_equal(colour.cpu().numpy(), ref_colour), call


def test_noalloc_after_a_setup_on_a_smaller_graph():
    # amg_setup launches the same colouring kernel on its own levels; a setup
    # of a small system between two calls on a larger graph must leave the
    # kernel able to take the larger graph
    big = P.stokes3d(16, 1)  # 4,913 nodes
    rp, ci, ref_colour, ref_nc = _level0_colours(big)
    lib = bamg.load()
    stream = torch.cuda.current_stream().cuda_stream
    colour, nc = _outputs(big.n_nodes)
    assert _call(lib, rp, ci, big.n_nodes, colour, nc, stream) == bamg.BAMG_OK
    _level0_colours(P.stokes2d(8, 1))  # 81 nodes
    colour2, nc2 = _outputs(big.n_nodes)
    assert _call(lib, rp, ci, big.n_nodes, colour2, nc2, stream) == bamg.BAMG_OK
    torch.cuda.synchronize()
    assert int(nc.item()) == ref_nc and int(nc2.item()) == ref_nc
    assert np.array_equal(colour.cpu().numpy(), ref_colour)
    assert np.array_equal(colour2.cpu().numpy(), ref_colour)


def test_noalloc_captured_in_a_graph_and_allocates_nothing():
    s = P.mhd2d(40, 2)
    rp, ci, ref_colour, ref_nc = _level0_colours(s)
    lib = bamg.load()
    colour, nc = _outputs(s.n_nodes)
    # a first call on this device (the address lookup), before any capture
    assert _call(lib, rp, ci, s.n_nodes, colour, nc, torch.cuda.current_stream().cuda_stream) == bamg.BAMG_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _call(lib, rp, ci, s.n_nodes, colour, nc, torch.cuda.current_stream().cuda_stream) == bamg.BAMG_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    colour.fill_(-7)
    nc.fill_(-7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = _call(lib, rp, ci, s.n_nodes, colour, nc, torch.cuda.current_stream().cuda_stream)
    assert st == bamg.BAMG_OK
    g.replay()
    torch.cuda.synchronize()
    assert int(nc.item()) == ref_nc
    assert np.array_equal(colour.cpu().numpy(), ref_colour)


def _with_extra_block(s, i, j):
    """The pattern of s with block (i, j) added to row i only (sorted)."""
    rp, ci = s.row_ptr.astype(np.int64), s.col_idx
    row = ci[rp[i]:rp[i + 1]]
    assert j not in row
    pos = rp[i] + int(np.searchsorted(row, j))
    ci2 = np.insert(ci, pos, j).astype(np.int32)
    rp2 = rp.copy()
    rp2[i + 1:] += 1
    return rp2.astype(np.int32), ci2


@pytest.mark.parametrize("side", ["lower_not_listed_back", "upper_not_listed_back"])
def test_noalloc_reports_a_one_sided_block(side):
    s = P.stokes2d(12, 1)
    n = s.n_nodes
    # node 40's row gains a far neighbour that does not list it back: below
    # it (node 2) or above it (node 150)
    i, j = (40, 2) if side == "lower_not_listed_back" else (40, 150)
    rp2, ci2 = _with_extra_block(s, i, j)
    lib = bamg.load()
    stream = torch.cuda.current_stream().cuda_stream
    colour, nc = _outputs(n)
    st = _call(lib, torch.from_numpy(rp2).cuda(), torch.from_numpy(ci2).cuda(), n, colour, nc, stream)
    assert st == bamg.BAMG_OK
    torch.cuda.synchronize()
    assert int(nc.item()) == -1
    # the symmetric pattern still colours on the next call (the shared
    # scratch keeps nothing that the next call depends on)
    rp, ci, ref_colour, ref_nc = _level0_colours(s)
    st = _call(lib, rp, ci, n, colour, nc, stream)
    torch.cuda.synchronize()
    assert st == bamg.BAMG_OK and int(nc.item()) == ref_nc
    assert np.array_equal(colour.cpu().numpy(), ref_colour)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = bamg.load()
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = lib.amg_colour_noalloc(d.data_ptr(), d.data_ptr(), 40001, d.data_ptr(), d.data_ptr(), None)
    assert st == bamg.BAMG_EUNSUPPORTED
