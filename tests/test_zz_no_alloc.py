"""The no-allocation cell sort against the run-based sort.

cpic_sort_cells_noalloc serves callers that cannot allocate device memory (code running
inside CUDA graph capture, hosts whose memory manager owns the whole device, loops that
must not pay for an allocation): it sorts caller-provided device arrays using scratch that
the library holds in a fixed device array. This test feeds it the same particles as a
run's own cpic_sort and checks that both produce the same live count, cell-ordered output
and the same set of particles (the order inside a cell is unspecified for both), on two
calls in a row, so that the second call sees the scratch the first one left behind.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1311_2286_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _records(cell, t, v):
    return np.sort(np.rec.fromarrays([cell, *t, v[0], v[1], v[2]]))


def _key(cell, n):
    idx = wl.unpack_cells(cell, len(n))
    key = np.zeros(cell.shape, np.int64)
    for a in reversed(range(len(n))):
        key = key * n[a] + idx[a]
    return key


def _valid(cell, n):
    """Slots in the grid: live (cell >= 0) with every axis index below its cell count."""
    idx = wl.unpack_cells(cell, len(n))
    ok = cell >= 0
    for a in range(len(n)):
        ok &= idx[a] < n[a]
    return ok


def _run_sort(cpic, w, s):
    run = cpic.run_from_workload(w)
    run.sort()
    out = run.particles(s)
    run.close()
    return out


def _noalloc_sort(cpic, ps, n):
    import torch

    D, cnt = len(n), ps.n
    dev = torch.device("cuda")
    cin = torch.from_numpy(ps.cell).to(dev)
    tin = torch.from_numpy(np.ascontiguousarray(ps.t).reshape(-1)).to(dev)
    vin = torch.from_numpy(np.ascontiguousarray(ps.v).reshape(-1)).to(dev)
    cout = torch.empty_like(cin)
    tout = torch.empty_like(tin)
    vout = torch.empty_like(vin)
    live = torch.zeros(1, dtype=torch.int64, device=dev)
    nn = (ctypes.c_int32 * 3)(n[0], n[1], n[2] if D == 3 else 1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cpic.check(cpic.load().cpic_sort_cells_noalloc(D, ctypes.cast(nn, ctypes.c_void_p), cnt, cpic._ptr(cin),
                                                   cpic._ptr(tin), cpic._ptr(vin), cpic._ptr(cout), cpic._ptr(tout),
                                                   cpic._ptr(vout), cpic._ptr(live), stream))
    torch.cuda.synchronize()
    m = int(live.item())
    cell = cout.cpu().numpy()[:m]
    t = tout.cpu().numpy().reshape(D, cnt)[:, :m]
    v = vout.cpu().numpy().reshape(3, cnt)[:, :m]
    return cell, t, v


def test_noalloc_sort_matches_run_sort_on_two_calls(cpic):
    """Three calls in a row (different particle sets: a 2D grid, a smaller 2D grid, a 3D
    grid), each compared with the run-based sort of the same input: equal live counts,
    non-decreasing cell keys, identical particle sets (bit for bit). Dead slots and, in 3D,
    packed cells beyond the grid's last plane are dropped by both (the run drops the latter
    when it loads them)."""
    cases = [
        wl.cylinder(n1=64, n2=128, npart_per_species=150_001, seed=21, inject=False),
        wl.cylinder(n1=32, n2=64, npart_per_species=70_007, seed=22, inject=False),
        wl.sphere(24, 20, 16, npart_per_species=60_013, seed=23),
    ]
    for w in cases:
        ps = w.particles[0]
        # dead slots in the input are dropped by both sorts
        ps.cell[::97] = -1
        if w.dim == 3:  # plane index n3 (inside the 10-bit field, outside the grid)
            ps.cell[5::101] = (ps.cell[5::101] & 0xFFFFF) | (w.n[2] << 20)
        ref = _run_sort(cpic, w, 0)
        got = _noalloc_sort(cpic, ps, w.n)
        assert got[0].shape == ref[0].shape == (int(np.sum(_valid(ps.cell, w.n))),)
        assert np.all(np.diff(_key(got[0], w.n)) >= 0)
        assert np.array_equal(_records(*got), _records(*ref))


def test_noalloc_sort_rejects_oversized_grid(cpic):
    nn = (ctypes.c_int32 * 3)(2048, 1024, 1)  # 2^21 cells > the fixed scratch
    live = ctypes.c_int64()
    st = cpic.load().cpic_sort_cells_noalloc(2, ctypes.cast(nn, ctypes.c_void_p), 0, None, None, None, None, None,
                                             None, ctypes.cast(ctypes.pointer(live), ctypes.c_void_p), None)
    assert st == cpic.CPIC_ERR_INVALID
    assert b"scratch" in cpic.load().cpic_last_error()
