"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes span several tiles and ragged tails (partial edge tiles, Gaussian counts
that are not multiples of the block size).  Tolerances: tile keys and sorted
lists bit-exact on identical FP32 inputs; images 1e-5 max-abs, leaving out only
pixels where a blend decision that FP32 rounding may flip could move the colour
or final T by more than half that (the oracle's flip bound; counted, under 5 %);
gradients 1e-4 relative per parameter group, and each entry within 1e-4 of the
mass of the sum that forms it (the sum of its terms' absolute values, which its
FP32 rounding scales with); z.Hz 1e-3 relative per group and of each entry's
mass; every entry plus the oracle's allowances: what the pixels where a
decision of its Gaussian's own (skip, cap, power sign, tile membership) or a
residual sign may flip in FP32 can change, and for z.Hz how far it moves when
the residuals move by their FP32 rounding (the L1 Gauss-Newton weight is that
sensitive near its floor); the TR update 1e-5 relative given identical inputs.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GROUPS = {"mean": slice(0, 3), "log_scale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "sh": slice(11, None)}


def _engine(n, deg, cams, tile=(16, 16), nu=1, **kw):
    from paper_2602_00395_gb300.engine import TRStep
    e = TRStep(n, deg, len(cams), cams[0].width, cams[0].height, nu=nu, tile=tile, **kw)
    e.set_cameras(cams)
    return e


def _cfg1():
    sc = S.make_scene(1000, 0, seed=1000, kind="cube", extent=1.0)
    return sc, [S.single_camera(128, 128)]


def _ragged():
    sc = S.make_scene(2999, 3, seed=1001, kind="cube", extent=1.0, log_scale_shift=math.log(1.5))
    cams = S.camera_ring(2, 97, 75, 1.0, seed=7, ring_factor=3.0)
    return sc, cams


def _records(e):
    return e.rec.view(e.V, e.n_pad, 12).cpu().numpy()


def _group_close(gpu, ref, tol, what, mass, *allowances, rnd=None):
    """Per parameter group: max |gpu - ref| <= tol max |ref|, and every entry
    within tol of the mass of its sum, both plus, entry by entry, the oracle's
    allowances for flips (arrays like ref, None for none); the per-entry check
    also admits `rnd`, the rounding the entry's terms carry."""
    sens = sum((a for a in allowances if a is not None), np.zeros_like(ref))
    rnd = np.zeros_like(ref) if rnd is None else rnd
    for name, sl in GROUPS.items():
        g, r, ms, se, rd = gpu[sl], ref[sl], mass[sl], sens[sl], rnd[sl]
        scale = np.abs(r).max()
        if scale == 0:
            assert np.abs(g).max() == 0, (what, name)
            continue
        err = np.abs(g - r)
        worst = (err - se).max() / scale
        assert worst <= tol, f"{what}/{name}: group relative error {worst:.3g} > {tol}"
        bad = err > tol * ms + se + rd
        assert not bad.any(), f"{what}/{name}: {int(bad.sum())} entries beyond {tol} of their mass"


# ------------------------------------------------------------------ project
@pytest.mark.parametrize("case", ["cfg1", "ragged"])
def test_project_matches_oracle(case):
    sc, cams = _cfg1() if case == "cfg1" else _ragged()
    e = _engine(sc.n, sc.sh_degree, cams, nu=2)
    e.set_params(sc.params)
    t = 3
    e.project(t, probes=True)
    torch.cuda.synchronize()
    rec = _records(e)
    tan = e.tan.view(e.V, e.n_pad, 1 + e.nu, 12).cpu().numpy()  # the record again, then its probes
    P = O.params64(sc)
    fields = [("mx", 0), ("my", 1), ("A", 2), ("B", 3), ("C", 4), ("o", 5), ("r", 6), ("g", 7), ("b", 8),
              ("depth", 9)]
    for v, cam in enumerate(cams):
        ref = O.project(P, sc.sh_degree, cam)
        valid = ref["valid"] > 0
        rad = rec[v, : sc.n, 10].view(np.int32)
        near_int = np.abs(ref["radius_raw"] - np.round(ref["radius_raw"])) < 1e-4 * ref["radius_raw"]
        assert np.array_equal((rad > 0), valid)
        assert np.all((rad == ref["radius"].astype(np.int32)) | near_int)
        for name, col in fields:
            g = rec[v, : sc.n, col][valid]
            r = ref[name][valid]
            scale = np.abs(r).max()
            np.testing.assert_allclose(g, r, rtol=2e-5, atol=2e-6 * scale, err_msg=name)
        # slot 0 of every (view, splat) in the tangent array is its record, bit for bit
        assert np.array_equal(tan[v, :, 0, :].view(np.uint32), rec[v].view(np.uint32))
        for k in range(e.nu):
            z = O.probe_matrix(42, t, k, e.rows, sc.n)
            rt = O.project_tangent(P, sc.sh_degree, cam, z)[valid]
            gt = tan[v, : sc.n, 1 + k, :9][valid]
            for q in range(9):
                scale = np.abs(rt[:, q]).max()
                assert np.abs(gt[:, q] - rt[:, q]).max() <= 1e-4 * scale + 1e-7, (k, q)
        # padding columns are culled
        assert np.all(rec[v, sc.n:, 10].view(np.int32) == 0)
        # the packed half-extents bound the alpha >= 1/255 footprint of the
        # record's own conic and opacity (computed here in FP64)
        A, B, C, o = (rec[v, : sc.n, c][valid].astype(np.float64) for c in (2, 3, 4, 5))
        ext = rec[v, : sc.n, 11][valid].view(np.uint32)
        hx = (ext & 0xFFFF).astype(np.uint16).view(np.float16).astype(np.float64)
        hy = (ext >> 16).astype(np.uint16).view(np.float16).astype(np.float64)
        tau = 2.0 * np.log(255.0 * o)
        det = A * C - B * B
        reach = tau > 1e-6
        assert np.all(np.isneginf(hx[tau < -1e-6])) and np.all(np.isneginf(hy[tau < -1e-6]))
        assert np.all(hx[reach] >= np.sqrt(tau[reach] * C[reach] / det[reach]))
        assert np.all(hy[reach] >= np.sqrt(tau[reach] * A[reach] / det[reach]))


# ------------------------------------------------------------------ bin/sort
def _tile_class(n):
    """8 floor(log2 n) + the next 3 bits of n, + 1 (0 for an empty list), at most 255."""
    n = np.asarray(n, np.int64)
    out = np.zeros(n.shape, np.int64)
    nz = n > 0
    e = np.floor(np.log2(n[nz])).astype(np.int64)
    m = np.where(e >= 3, (n[nz] >> np.maximum(e - 3, 0)) & 7, (n[nz] << np.maximum(3 - e, 0)) & 7)
    out[nz] = np.minimum(255, 1 + 8 * e + m)
    return out


def _write_records(e, mx, my, r, d, ext, conic):
    rec = torch.zeros(e.V, e.n_pad, 12, dtype=torch.float32)
    n = mx.shape[1]
    rec[:, :n, 0] = torch.from_numpy(mx)
    rec[:, :n, 1] = torch.from_numpy(my)
    for k in range(3):
        rec[:, :n, 2 + k] = torch.from_numpy(np.ascontiguousarray(conic[k]))
    rec[:, :n, 9] = torch.from_numpy(d)
    rec[:, :n, 10] = torch.from_numpy(r.astype(np.int32).view(np.float32))
    rec[:, :n, 11] = torch.from_numpy(ext.astype(np.uint32).view(np.float32))
    e.rec.copy_(rec.reshape(-1).to(e.device))


@pytest.mark.parametrize("W,H,tile,V,n,maxr,box", [
    (128, 128, (16, 16), 1, 1000, 40, True),
    (128, 128, (16, 16), 1, 1000, 40, False),
    (97, 53, (16, 8), 3, 4001, 30, True),
    (61, 45, (8, 8), 2, 777, 60, False),
    (97, 53, (32, 16), 3, 4001, 30, True),  # 512-pixel tiles: blocks of eight warps
    (1297, 840, (16, 32), 2, 150000, 80, False),
    (1297, 840, (16, 16), 2, 150000, 80, True),  # ~ millions of pairs, many chunks
    (1297, 840, (16, 16), 2, 150000, 80, False),
    # more tiles per view than the shared counters hold: pairs sorted by radix passes
    (3840, 2160, (16, 16), 1, 60000, 120, True),
    (2100, 1500, (8, 8), 2, 30000, 40, False),
])
def test_bin_sort_bit_exact(W, H, tile, V, n, maxr, box):
    """Keys, values and ranges equal the oracle's from the same FP32 records, with
    the 3DGS tile square (box False) and with it narrowed to the footprint box."""
    recs = [S.projected_records(n, W, H, seed=100 + v, max_radius=maxr) for v in range(V)]
    mx = np.stack([a[0] for a in recs]); my = np.stack([a[1] for a in recs])
    r = np.stack([a[2] for a in recs]); d = np.stack([a[3] for a in recs])
    ext = np.stack([a[4] for a in recs])
    conic = np.stack([a[5] for a in recs], axis=1)  # 3 x V x n
    keys, vals, ranges = O.bin_sort(mx, my, r, d, W, H, *tile, extents=ext if box else None, conic=conic)
    cams = [S.single_camera(W, H)] * V
    e = _engine(n, 0, cams, tile=tile, nu=0, capacity=len(keys) + 123, footprint_bins=box)
    _write_records(e, mx, my, r, d, ext, conic)
    e.bin_sort()
    torch.cuda.synchronize()
    P = int(e.n_pairs.item())
    assert P == len(keys)
    assert e.read_status() == 0
    # the device keys are the tile halves of the oracle's (tile, depth) keys; the
    # depth order within a tile is the order of the splat indices compared next
    np.testing.assert_array_equal(e.keys[:P].cpu().numpy().view(np.uint32), (keys >> np.uint64(32)).astype(np.uint32))
    np.testing.assert_array_equal(e.vals[:P].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(e.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2), ranges)
    # the blends' tile order: every tile once, list lengths by class heaviest first
    order = e.order.cpu().numpy().view(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(len(order)))
    cls = _tile_class(ranges[:, 1].astype(np.int64) - ranges[:, 0])
    assert np.all(np.diff(cls[order]) <= 0)


@pytest.mark.parametrize("W,H", [(128, 96), (3840, 2160)])
def test_bin_sort_capacity_overflow_is_flagged_and_in_bounds(W, H):
    n = 3000
    mx, my, r, d, ext, conic = S.projected_records(n, W, H, seed=5, max_radius=50)
    keys, _, _ = O.bin_sort(mx, my, r, d, W, H, extents=ext, conic=conic)
    e = _engine(n, 0, [S.single_camera(W, H)], nu=0, capacity=len(keys) // 3)
    _write_records(e, mx[None], my[None], r[None], d[None], ext[None], conic[:, None])
    e.bin_sort()
    torch.cuda.synchronize()
    from paper_2602_00395_gb300 import gs3dtr as G
    assert int(e.n_pairs.item()) == len(keys)
    assert e.read_status() & G.GS_FLAG_CAPACITY
    cap = len(keys) // 3
    rg = e.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert rg.max() <= cap


@pytest.mark.parametrize("W,H,maxr", [(1297, 840, 120), (256, 256, 60)])
def test_bin_sort_far_past_capacity_keeps_every_slot_in_range(W, H, maxr):
    """Pairs far beyond the capacity (some records' row tables do not fit either):
    the overflow is flagged, the pair count is the need, and every stored pair and
    range is in range, so that later calls read nothing out of bounds."""
    n = 20000
    mx, my, r, d, ext, conic = S.projected_records(n, W, H, seed=17, max_radius=maxr)
    keys, _, _ = O.bin_sort(mx, my, r, d, W, H, extents=ext, conic=conic)
    cap = 64
    e = _engine(n, 0, [S.single_camera(W, H)], nu=0, capacity=cap)
    _write_records(e, mx[None], my[None], r[None], d[None], ext[None], conic[:, None])
    e.bin_sort()
    torch.cuda.synchronize()
    from paper_2602_00395_gb300 import gs3dtr as G
    assert int(e.n_pairs.item()) == len(keys) > 100 * cap
    assert e.read_status() & G.GS_FLAG_CAPACITY
    k = e.keys[:cap].cpu().numpy().view(np.uint32)
    v = e.vals[:cap].cpu().numpy().view(np.uint32)
    assert np.all(k < e.Tx * e.Ty) and np.all(v < n)
    rg = e.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert rg.max() <= cap


def test_bin_sort_empty_input():
    W, H, n = 64, 64, 100
    e = _engine(n, 0, [S.single_camera(W, H)], nu=0, capacity=1024)
    e.rec.zero_()
    e.bin_sort()
    torch.cuda.synchronize()
    assert int(e.n_pairs.item()) == 0
    assert int(e.ranges.abs().sum().item()) == 0


# ------------------------------------------------------------------ forward
def _render_compare(sc, cams, tile=(16, 16), box=True, batch=0):
    e = _engine(sc.n, sc.sh_degree, cams, tile=tile, nu=0, footprint_bins=box, batch=batch)
    e.set_params(sc.params)
    e.ensure_capacity()
    e.render()
    torch.cuda.synchronize()
    with O.footprint_bins(box):
        ref = O.render(O.params64(sc), sc.sh_degree, cams, *tile)
    V, H, W = len(cams), cams[0].height, cams[0].width
    img = e.image.view(V, 3, H, W).cpu().numpy()
    T = e.final_T.view(V, H, W).cpu().numpy()
    nc = e.n_contrib.view(V, H, W).cpu().numpy()
    ok = (ref["impact"] <= 5e-6) & (ref["t_impact"] <= 5e-6)
    # a pixel where a decision FP32 may flip could move the value by more than
    # half the tolerance must equal one of the results the blend reaches when
    # those decisions go either way; it is left out only where they are not
    # resolved (more than 64, or small flips summing past half the tolerance)
    unresolved = np.zeros_like(ok)
    for v in range(V):
        ys, xs = np.nonzero(~ok[v])
        if len(xs) == 0:
            continue
        with O.footprint_bins(box):
            px = O.render_pixels(O.params64(sc), sc.sh_degree, cams[v], xs, ys, tw=tile[0], th=tile[1],
                                 outcomes=64)
        res, matched, _ = O.match_outcomes(px, img[v][:, ys, xs].T, T[v][ys, xs], img_tol=1e-5, flip_max=5e-6)
        assert np.all(matched[res]), [(int(xs[q]), int(ys[q])) for q in np.nonzero(res & ~matched)[0][:8]]
        in_range = (nc[v][ys, xs] >= px["n_contrib_lo"]) & (nc[v][ys, xs] <= px["n_contrib_hi"])
        assert np.all(in_range[res])
        unresolved[v][ys[~res], xs[~res]] = True
    return e, ref, img, T, nc, ok, unresolved


@pytest.mark.parametrize("case,tile,box,batch", [("cfg1", (16, 16), True, 0), ("cfg1", (16, 16), False, 0),
                                                ("ragged", (16, 8), True, 0), ("ragged", (8, 8), True, 0),
                                                ("ragged", (16, 16), False, 0), ("ragged", (16, 16), True, 32),
                                                ("cfg1", (16, 16), True, 512), ("ragged", (32, 16), True, 0),
                                                ("ragged", (16, 32), False, 0), ("cfg1", (32, 16), True, 128)])
def test_raster_fwd_matches_oracle(case, tile, box, batch):
    """Image, final T, n_contrib and the pair count equal the oracle's, binning by
    the footprint (box True) or by the whole 3DGS tile square, with the default
    and other per-block record batches."""
    sc, cams = _cfg1() if case == "cfg1" else _ragged()
    e, ref, img, T, nc, ok, unresolved = _render_compare(sc, cams, tile, box, batch)
    assert int(e.n_pairs.item()) == ref["n_pairs"] or (~ok).any()
    # every pixel is compared: those a flip may move by more than half the
    # tolerance against the oracle's outcomes (in _render_compare), the rest here
    print(f"\n{case} {tile} box={box} batch={batch}: {1.0 - ok.mean():.3%} of pixels compared with the "
          f"flip outcomes, {int(unresolved.sum())} unresolved")
    assert unresolved.mean() < 1e-4, unresolved.mean()
    err = np.abs(img - ref["image"]).max(axis=1)[ok]
    assert err.max() <= 1e-5, err.max()
    assert np.abs(T - ref["final_T"])[ok].max() <= 1e-5
    # n_contrib within the range that tile sets within rounding give (equal to
    # the oracle's wherever no such tile set is in front of the last blend)
    in_range = (nc >= ref["n_contrib_lo"]) & (nc <= ref["n_contrib_hi"])
    assert np.all(in_range[ok])
    assert np.mean((nc == ref["n_contrib"])[ok]) >= 0.95


# ------------------------------------------------------------------ reverse
def _grad_case(case, nu, loss_kind=0, batch=0, tile=(16, 16)):
    sc, cams = _cfg1() if case == "cfg1" else _ragged()
    V, H, W = len(cams), cams[0].height, cams[0].width
    target = S.noise_target(V, H, W, seed=2000)
    e = _engine(sc.n, sc.sh_degree, cams, tile=tile, nu=nu, loss_kind=loss_kind, batch=batch)
    e.set_params(sc.params)
    e.set_target(target)
    e.ensure_capacity()
    t = 4
    e.project(t, probes=nu > 0)
    e.bin_sort()
    e.raster_fwd(t, probes=nu > 0)
    e.loss_val.zero_()
    e.raster_bwd(t, probes=nu > 0)
    torch.cuda.synchronize()
    ref = O.backward(O.params64(sc), sc.sh_degree, cams, target.astype(np.float64), loss_kind=loss_kind,
                     seed=42, t=t, nu=nu, tw=tile[0], th=tile[1], want_tangents=nu > 0, masses=True)
    return sc, e, ref


@pytest.mark.parametrize("case,nu,loss_kind,batch,tile", [("cfg1", 0, 0, 0, (16, 16)), ("cfg1", 1, 0, 0, (16, 16)),
                                                          ("ragged", 2, 0, 0, (16, 16)), ("ragged", 1, 1, 0, (16, 16)),
                                                          ("ragged", 2, 0, 64, (16, 16)),
                                                          ("cfg1", 1, 0, 512, (16, 16)),
                                                          ("ragged", 2, 0, 0, (32, 16)),
                                                          ("cfg1", 1, 1, 0, (16, 32))])
def test_gradient_and_hutchinson_match_oracle(case, nu, loss_kind, batch, tile):
    sc, e, ref = _grad_case(case, nu, loss_kind, batch, tile)
    grad = e.grad[:, : sc.n].cpu().numpy()
    _group_close(grad, ref["grad"], 1e-4, "grad", ref["grad_mass"], ref["grad_allow"], rnd=ref["grad_round"])
    assert abs(float(e.loss_val.item()) - ref["loss"]) <= 1e-5 * ref["loss"]
    if nu:
        hz = e.hz[:, : sc.n].cpu().numpy()
        _group_close(hz, ref["hz"], 1e-3, "hz", ref["hz_mass"], ref["hz_sens"], ref["hz_allow"], rnd=ref["hz_round"])
        V, H, W = e.V, e.H, e.W
        it = e.image_tan.view(nu, V, 3, H, W).cpu().numpy()
        scale = np.abs(ref["image_tangent"]).max()
        assert np.abs(it - ref["image_tangent"]).max() <= 1e-4 * scale


@pytest.mark.parametrize("tile,box", [((16, 16), True), ((16, 16), False), ((32, 16), True)])
def test_reverse_pass_with_the_forward_masks_equals_its_own_footprint_test(tile, box):
    """The reverse pass reads the forward pass's block masks (gs_sorted.masks)
    or, given none, tests each splat's footprint against its warp's block
    itself: the same splats are visited, so the gradient and Hutchinson rows
    agree up to the order of the float atomics that sum them."""
    sc, cams = _ragged()
    V, H, W = len(cams), cams[0].height, cams[0].width
    e = _engine(sc.n, sc.sh_degree, cams, tile=tile, nu=2, footprint_bins=box)
    e.set_params(sc.params)
    e.set_target(S.noise_target(V, H, W, seed=2000))
    e.ensure_capacity()
    t = 3
    e.project(t)
    e.bin_sort()
    e.raster_fwd(t)
    assert e.masks_valid
    out = []
    for use_masks in (True, False):
        e.grad.zero_()
        e.hz.zero_()
        e.masks_valid = use_masks
        e.raster_bwd(t)
        torch.cuda.synchronize()
        out.append((e.grad[:, : sc.n].cpu().numpy().copy(), e.hz[:, : sc.n].cpu().numpy().copy()))
    assert e.read_status() == 0
    for a, b in zip(out[0], out[1]):
        assert np.abs(a).max() > 0
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_step_with_separate_curvature_batch_matches_oracle():
    """Algorithm 1 with S2 != S1 (Sec. 4.1): the gradient from S1's view, the
    Hutchinson product from S2's view, then the update; l = 2 so that the next
    step takes no curvature and keeps d_ema."""
    from paper_2602_00395_gb300.engine import TRConfig
    sc, cams2 = _ragged()
    s1, s2 = [cams2[0]], [cams2[1]]
    H, W = s1[0].height, s1[0].width
    tg = S.noise_target(2, H, W, seed=2001)
    e = _engine(sc.n, sc.sh_degree, s1, nu=2, cfg=TRConfig(l=2))
    e.set_params(sc.params)
    e.set_target(tg[:1])
    from paper_2602_00395_gb300 import gs3dtr as G
    cams_s2 = torch.from_numpy(G.camera_bytes(s2)).cuda()
    tg_s2 = torch.from_numpy(tg[1:].reshape(-1)).cuda()
    e.ensure_capacity()
    e.cams, c1 = cams_s2, e.cams
    e.ensure_capacity()
    e.cams = c1
    t, eps = 1, 1e-6
    e.step_s2(t, eps, cams_s2, tg_s2)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    P = O.params64(sc)
    r1 = O.backward(P, sc.sh_degree, s1, tg[:1].astype(np.float64), seed=42, t=t, nu=2, masses=True)
    r2 = O.backward(P, sc.sh_degree, s2, tg[1:].astype(np.float64), seed=42, t=t, nu=2, masses=True)
    _group_close(e.grad[:, : sc.n].cpu().numpy(), r1["grad"], 1e-4, "grad(S1)", r1["grad_mass"], r1["grad_allow"],
                 rnd=r1["grad_round"])
    _group_close(e.hz[:, : sc.n].cpu().numpy(), r2["hz"], 1e-3, "hz(S2)", r2["hz_mass"], r2["hz_sens"],
                 r2["hz_allow"], rnd=r2["hz_round"])
    d1 = e.d_ema.clone()
    e.step_s2(2, eps, cams_s2, tg_s2)  # (2 - 1) % 2 != 0: no curvature, d_ema kept
    torch.cuda.synchronize()
    assert torch.equal(e.d_ema, d1)


@pytest.mark.parametrize("want_grad", [True, False])
def test_reverse_pass_from_given_cotangents_matches_oracle(want_grad):
    """GS_LOSS_COTANGENT: with dL/dC = c and u_k = (1/m) J z_k the reverse pass
    gives J^T c and the Hutchinson diagonal of (1/m) J^T J, which the oracle
    computes as the L2 objective of the target image - m c."""
    sc, cams = _ragged()
    V, H, W, nu, t = len(cams), cams[0].height, cams[0].width, 2, 6
    e = _engine(sc.n, sc.sh_degree, cams, nu=nu)
    e.set_params(sc.params)
    e.ensure_capacity()
    e.project(t, probes=True)
    e.bin_sort()
    e.raster_fwd(t, probes=True)
    P = O.params64(sc)
    img = O.render(P, sc.sh_degree, cams, with_margin=False)["image"]
    m = 3 * H * W * V
    c = np.random.default_rng(3).normal(size=img.shape) * (1.0 / m)
    ref = O.backward(P, sc.sh_degree, cams, img - m * c, loss_kind=1, seed=42, t=t, nu=nu, want_tangents=True,
                     masses=True)
    streams = ([c] if want_grad else []) + [ref["image_tangent"][k] / m for k in range(nu)]
    cot = torch.from_numpy(np.stack(streams).astype(np.float32).reshape(-1)).cuda()
    e.raster_bwd_cotangent(cot, t, want_grad)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    if want_grad:
        _group_close(e.grad[:, : sc.n].cpu().numpy(), ref["grad"], 1e-4, "grad", ref["grad_mass"], ref["grad_allow"],
                     rnd=ref["grad_round"])
    _group_close(e.hz[:, : sc.n].cpu().numpy(), ref["hz"], 1e-3, "hz", ref["hz_mass"], ref["hz_allow"],
                 rnd=ref["hz_round"])


def test_reverse_workspace_is_left_clear_and_reused():
    """The reverse call leaves its cotangent rows zero and says so in the
    workspace header, so the next call skips clearing them; a workspace of
    arbitrary bytes is cleared first.  Either way the results are the first
    call's (up to the order of the float atomics)."""
    sc, e, ref = _grad_case("ragged", 2)
    g1, h1 = e.grad[:, : sc.n].clone(), e.hz[:, : sc.n].clone()
    ws = e.bwd_ws
    hdr = ws[:16].cpu().numpy().view(np.uint64)
    rows = ws[256:].view(torch.float32)
    assert hdr[0] == 0x9D2C5680A3B1F4E7 and hdr[1] >= rows.numel() and int(torch.count_nonzero(rows)) == 0

    def again():
        e.loss_val.zero_()
        e.raster_bwd(4, probes=True)
        torch.cuda.synchronize()
        assert e.read_status() == 0
        for a, b in ((e.grad[:, : sc.n], g1), (e.hz[:, : sc.n], h1)):
            torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6 * b.abs().max().item())

    again()                      # rows known clear: nothing cleared
    ws.fill_(0x7F)               # foreign bytes, header included
    again()
    e.hvp_diag(4)                # fewer streams over the same workspace
    torch.cuda.synchronize()
    again()
    assert int(torch.count_nonzero(rows)) == 0


def test_hvp_diag_standalone_equals_fused():
    sc, e, ref = _grad_case("cfg1", 1)
    fused = e.hz.clone()
    e.hz.fill_(123.0)
    e.hvp_diag(4)
    torch.cuda.synchronize()
    np.testing.assert_allclose(e.hz[:, : sc.n].cpu().numpy(), fused[:, : sc.n].cpu().numpy(), rtol=1e-5,
                               atol=1e-6 * fused.abs().max().item())


# ------------------------------------------------------------------ update
@pytest.mark.parametrize("deg,t,l,mean_exact", [(0, 1, 10, 0), (3, 1, 1, 1), (3, 5, 2, 0), (1, 2, 3, 0)])
def test_tr_update_matches_oracle(deg, t, l, mean_exact):
    from paper_2602_00395_gb300.engine import TRConfig
    n = 5003
    sc = S.make_scene(n, deg, seed=77)
    rng = np.random.default_rng(t + 10 * deg)
    rows = sc.params.shape[0]
    P32 = sc.params.copy()
    P32[10, :n] = rng.normal(0, 4, n)  # includes alpha <= eps Gaussians
    ge = (rng.normal(size=P32.shape) * 1e-3).astype(np.float32)
    de = np.abs(rng.normal(size=P32.shape) * 1e-2).astype(np.float32)
    de[:, ::7] = 0.0  # exercises the d_floor
    g = (rng.normal(size=P32.shape) * 1e-3).astype(np.float32)
    hz = (rng.normal(size=P32.shape) * 1e-2).astype(np.float32)
    cfg = TRConfig(l=l, mean_exact=mean_exact)
    eps = 1e-6 * (1e-2) ** ((t - 1) / 9)
    e = _engine(n, deg, [S.single_camera(64, 64)], nu=1, cfg=cfg)
    e.x.copy_(torch.from_numpy(P32)); e.g_ema.copy_(torch.from_numpy(ge)); e.d_ema.copy_(torch.from_numpy(de))
    e.grad.copy_(torch.from_numpy(g)); e.hz.copy_(torch.from_numpy(hz))
    eta = torch.zeros_like(e.x)
    e.update(t, eps, with_hz=True, eta_out=eta)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    f32 = lambda v: float(np.float32(v))  # the hyper-parameters the kernel receives
    ocfg = O.tr_config(theta1=f32(cfg.theta1), theta2=f32(cfg.theta2), d_floor=f32(cfg.d_floor),
                       color_floor=f32(cfg.color_floor), l=l, mean_exact=mean_exact)
    rx, rg, rd, reta = O.tr_update(P32[:, :n], ge[:, :n], de[:, :n], g[:, :n], hz[:, :n], deg, t=t, eps=np.float32(eps),
                                   cfg=ocfg)
    # FP32 evaluates a x + b y with an error of a few ulps of |a x| + |b y|,
    # so tolerances scale with the operands, not with the (cancelling) result
    a1, a2 = f32(cfg.theta1), f32(cfg.theta2)
    g_scale = a1 * np.abs(ge[:, :n]) + (1 - a1) * np.abs(g[:, :n])
    d_scale = a2 * np.abs(de[:, :n]) + (1 - a2) * np.abs(hz[:, :n])
    hvp_step = (t - 1) % l == 0
    if not hvp_step:
        d_scale = np.abs(de[:, :n])
    ge_gpu = e.g_ema[:, :n].cpu().numpy().astype(np.float64)
    de_gpu = e.d_ema[:, :n].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(ge_gpu - rg) <= 1e-6 * g_scale + 1e-30)
    assert np.all(np.abs(de_gpu - rd) <= 1e-6 * d_scale + 1e-30)
    eg = eta[:, :n].cpu().numpy()
    fin = np.isfinite(reta)
    assert np.array_equal(np.isfinite(eg), fin)
    np.testing.assert_allclose(eg[fin], reta[fin], rtol=1e-5)
    # the step x_{t+1} - x_t: clipped steps equal +-eta (1e-5 relative); unclipped
    # ones inherit the operand-scaled error of g_ema / max(d_ema, d_floor)
    den = np.maximum(rd, cfg.d_floor)
    step_scale = np.minimum(np.where(fin, reta, np.inf), (g_scale + np.abs(rg) * d_scale / den) / den)
    dx_gpu = e.x[:, :n].cpu().numpy().astype(np.float64) - P32[:, :n]
    dx_ref = rx - P32[:, :n].astype(np.float64)
    ulp = np.spacing(np.abs(e.x[:, :n].cpu().numpy())).astype(np.float64)
    assert np.all(np.abs(dx_gpu - dx_ref) <= 1e-5 * step_scale + 2 * ulp)
    # some steps are clipped and some are not
    clipped = np.isclose(np.abs(dx_ref), np.where(fin, reta, -1), rtol=1e-12)
    assert clipped.any() and (~clipped).any()


@pytest.mark.parametrize("deg,t", [(3, 1), (1, 7)])
def test_adam_tr_update_matches_oracle(deg, t):
    """ADAM-TR (Sec. 5): the Adam step clipped by the trust region, vs the oracle."""
    from paper_2602_00395_gb300 import gs3dtr as G
    n = 4001
    sc = S.make_scene(n, deg, seed=91)
    rng = np.random.default_rng(t)
    P32 = sc.params.copy()
    m = (rng.normal(size=P32.shape) * 1e-3).astype(np.float32)
    v = (np.abs(rng.normal(size=P32.shape)) * 1e-6).astype(np.float32)
    g = (rng.normal(size=P32.shape) * 1e-3).astype(np.float32)
    eps = 1e-6
    e = _engine(n, deg, [S.single_camera(64, 64)], nu=0)
    e.x.copy_(torch.from_numpy(P32)); e.g_ema.copy_(torch.from_numpy(m)); e.d_ema.copy_(torch.from_numpy(v))
    e.grad.copy_(torch.from_numpy(g))
    adam = G.adam_struct()
    eta = torch.zeros_like(e.x)
    e.update_adam(t, eps, adam, eta)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    f32 = lambda a: np.float64(np.float32(a))  # the hyper-parameters the kernel receives
    oadam = O.adam_config(f32(adam.beta1), f32(adam.beta2), f32(adam.eps_adam), [f32(x) for x in adam.lr])
    ocfg = O.tr_config(theta1=f32(e.cfg.theta1), theta2=f32(e.cfg.theta2), d_floor=f32(e.cfg.d_floor),
                       color_floor=f32(e.cfg.color_floor), l=e.cfg.l, mean_exact=e.cfg.mean_exact)
    rx, rm, rv, reta = O.adam_tr_update(P32[:, :n], m[:, :n], v[:, :n], g[:, :n], deg, t=t, eps=np.float32(eps),
                                        cfg=ocfg, adam=oadam)
    mg = e.g_ema[:, :n].cpu().numpy().astype(np.float64)
    vg = e.d_ema[:, :n].cpu().numpy().astype(np.float64)
    b1, b2 = f32(adam.beta1), f32(adam.beta2)
    assert np.all(np.abs(mg - rm) <= 1e-6 * (b1 * np.abs(m[:, :n]) + (1 - b1) * np.abs(g[:, :n])) + 1e-30)
    assert np.all(np.abs(vg - rv) <= 1e-6 * (b2 * np.abs(v[:, :n]) + (1 - b2) * g[:, :n] ** 2) + 1e-30)
    eg = eta[:, :n].cpu().numpy()
    fin = np.isfinite(reta)
    assert np.array_equal(np.isfinite(eg), fin)
    np.testing.assert_allclose(eg[fin], reta[fin], rtol=1e-5)
    # x moves by the clipped step: at most the radius, and the Adam step where unclipped
    dx_gpu = e.x[:, :n].cpu().numpy().astype(np.float64) - P32[:, :n]
    dx_ref = rx - P32[:, :n]
    tol = 1e-4 * np.abs(dx_ref) + 2e-7 * np.abs(P32[:, :n]) + 1e-12
    assert np.all(np.abs(dx_gpu - dx_ref) <= tol)


@pytest.mark.parametrize("case,nu", [("cfg1", 1), ("ragged", 2)])
def test_dssim_gradient_and_hutchinson_match_oracle(case, nu):
    """The D-SSIM pixel loss (Eq. pixel_loss, lambda = 0.2): objective, gradient and
    Hutchinson diagonal through gs_dssim_cotangents and the reverse pass."""
    sc, cams = _cfg1() if case == "cfg1" else _ragged()
    V, H, W = len(cams), cams[0].height, cams[0].width
    target = S.smooth_target(V, H, W, seed=2002)
    e = _engine(sc.n, sc.sh_degree, cams, nu=nu, dssim_lambda=0.2)
    e.set_params(sc.params)
    e.set_target(target)
    e.ensure_capacity()
    t = 5
    e.loss_val.zero_()
    e.project(t, probes=True)
    e.bin_sort()
    e.raster_fwd(t, probes=True)
    e.raster_bwd(t, probes=True)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    ref = O.backward(O.params64(sc), sc.sh_degree, cams, target.astype(np.float64), loss_kind=2, lam=0.2, seed=42,
                     t=t, nu=nu, masses=True)
    assert abs(float(e.loss_val.item()) - ref["loss"]) <= 1e-5 * ref["loss"]
    _group_close(e.grad[:, : sc.n].cpu().numpy(), ref["grad"], 1e-4, "grad", ref["grad_mass"], ref["grad_allow"],
                 rnd=ref["grad_round"])
    _group_close(e.hz[:, : sc.n].cpu().numpy(), ref["hz"], 1e-3, "hz", ref["hz_mass"], ref["hz_allow"],
                 rnd=ref["hz_round"])
    fused = e.hz.clone()
    e.hz.fill_(7.0)
    e.hvp_diag(t)
    torch.cuda.synchronize()
    np.testing.assert_allclose(e.hz[:, : sc.n].cpu().numpy(), fused[:, : sc.n].cpu().numpy(), rtol=1e-5,
                               atol=1e-6 * fused.abs().max().item())
