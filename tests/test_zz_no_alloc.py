"""gs_bin_sort_noalloc: the bin/sort for callers that cannot allocate.

Callers whose allocator is frozen (a server that reserved its memory at start),
plugins that only receive device pointers, or loops that must avoid cudaMalloc's
synchronisation cannot hand gs_bin_sort a workspace; gs_bin_sort_noalloc takes
its scratch from a fixed device array inside the library.  Its output must equal
gs_bin_sort's (bit-exact, as for every integer output) on two calls in a row,
the second with a different, smaller input so that stale scratch from the first
call cannot leak into it.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _records_into(e, n, W, H, V, seed, max_radius):
    recs = [S.projected_records(n, W, H, seed=seed + v, max_radius=max_radius) for v in range(V)]
    rec = torch.zeros(V, e.n_pad, 12, dtype=torch.float32)
    for v, (mx, my, r, d, ext, conic) in enumerate(recs):
        rec[v, :n, 0] = torch.from_numpy(mx)
        rec[v, :n, 1] = torch.from_numpy(my)
        for k in range(3):
            rec[v, :n, 2 + k] = torch.from_numpy(np.ascontiguousarray(conic[k]))
        rec[v, :n, 9] = torch.from_numpy(d)
        rec[v, :n, 10] = torch.from_numpy(r.astype(np.int32).view(np.float32))
        rec[v, :n, 11] = torch.from_numpy(ext.view(np.float32))
    e.rec.copy_(rec.reshape(-1).to(e.device))


def _outputs(e):
    P = int(e.n_pairs.item())
    return (P, e.keys[:P].cpu().numpy().copy(), e.vals[:P].cpu().numpy().copy(), e.ranges.cpu().numpy().copy())


def test_noalloc_sort_equals_workspace_sort_on_two_calls():
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import TRStep
    L = G.load()
    W, H, V = 311, 197, 2
    for call, (n, seed, max_r) in enumerate(((20000, 700, 40), (5001, 900, 25))):
        e = TRStep(n, 0, V, W, H, nu=0, capacity=1 << 20)
        e.set_cameras([S.single_camera(W, H)] * V)
        _records_into(e, n, W, H, V, seed, max_r)
        e.bin_sort()  # the existing entry point with its caller workspace
        torch.cuda.synchronize()
        P, keys, vals, ranges = _outputs(e)
        assert P > 10000 and e.read_status() == 0
        e.keys.fill_(-1)
        e.vals.fill_(-1)
        e.ranges.fill_(-1)
        e.n_pairs.fill_(-1)
        rc = L.gs_bin_sort_noalloc(C.byref(e.proj()), e.n_pad, e.frame, C.byref(e.sorted()),
                                   G.ptr(e.status), G.stream_handle())
        assert rc == G.GS_OK, L.gs_last_error()
        torch.cuda.synchronize()
        P2, keys2, vals2, ranges2 = _outputs(e)
        assert e.read_status() == 0, call
        assert P2 == P, call
        np.testing.assert_array_equal(keys2, keys)
        np.testing.assert_array_equal(vals2, vals)
        np.testing.assert_array_equal(ranges2, ranges)


def test_noalloc_sort_rejects_requests_beyond_its_scratch():
    from paper_2602_00395_gb300 import gs3dtr as G
    L = G.load()
    frame = G.frame_struct(8, 1920, 1080)
    assert G.gs_bin_sort_workspace_size(1 << 20, frame, 50_000_000) > (32 << 20)
    proj = G.gs_projected(16, 16)  # never dereferenced: the size check comes first
    out = G.gs_sorted(16, 16, 16, 16, 50_000_000)
    rc = L.gs_bin_sort_noalloc(C.byref(proj), 1 << 20, frame, C.byref(out), None, None)
    assert rc == G.GS_ERR_INVALID_ARG
    assert b"scratch" in L.gs_last_error()
