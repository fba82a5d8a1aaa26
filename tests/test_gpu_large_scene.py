"""The large-scene configuration: 6M Gaussians (SH degree 3, the 20-cluster
generator), one 1920x1080 view per step, one probe, the step's backward and
Hutchinson product through torch.autograd.

The render is `autograd.render`; the L1 objective of Sec. 3.2 is formed in
PyTorch on its output, and `loss.backward()` runs the reverse pass from the
image gradient (recomputing each T_i from the final T: nothing per pair is kept
between the passes).  The Gauss-Newton diagonal comes from `gn_diagonal` with
the L1 weights 1/(4 max(|r|, delta))/m, which the library applies to J z_k
itself.  Compared with the FP64 oracle on what it computes one by one, with the
readings of the benchmark-size test:
  * 256 sampled pixels: colour and final T (1e-5), n_contrib in the range the
    oracle's flip analysis allows, leaving out pixels where a decision FP32 may
    flip could move the colour or final T by more than half the tolerance;
  * 64 sampled Gaussians: gradient rows (1e-4 of the group's largest sampled
    entry, each entry within 1e-4 of its sum's mass) and Hutchinson rows (1e-3
    of the group's largest, plus the oracle's bound on how far an entry moves
    when the residuals move by their FP32 rounding), unless their own decisions
    are within rounding of flipping.
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, W, H, DEG = 6_000_000, 1920, 1080, 3
GROUPS = {"mean": slice(0, 3), "log_scale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "sh": slice(11, None)}


@pytest.fixture(scope="module")
def large():
    from paper_2602_00395_gb300.autograd import gn_diagonal, render
    from paper_2602_00395_gb300.engine import TRConfig, TRStep
    sc = S.make_scene(N, DEG, seed=1004, kind="clusters", extent=10.0)
    cam = S.camera_ring(64, W, H, 10.0, seed=7)[5]
    target = S.smooth_target(1, H, W, seed=2004)
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    e = TRStep(N, DEG, 1, W, H, nu=1, cfg=TRConfig(l=1))
    e.set_cameras([cam])
    e.set_params(sc.params)
    e.ensure_capacity()
    t = 3
    tg = torch.from_numpy(target).cuda()
    m = 3 * H * W
    params = e.x.clone().requires_grad_(True)
    img = render(params, e)
    loss = (img - tg).abs().sum() / (2 * m)
    loss.backward()
    r = (img.detach() - tg)
    w = 1.0 / (4.0 * torch.clamp(r.abs(), min=1e-3)) / m
    hz = gn_diagonal(params, w, e, t)
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated()
    assert e.read_status() == 0
    out = dict(sc=sc, cam=cam, target=target, t=t, img=img.detach()[0].cpu().numpy(),
               final_T=e.final_T.view(H, W).cpu().numpy(), n_contrib=None, grad=params.grad[:, :N].cpu().numpy(),
               hz=hz[:, :N].cpu().numpy(),
               peak=peak, state_bytes=5 * e.rows * e.n_pad * 4, loss=float(loss.detach()))
    # n_contrib of the plain render (gn_diagonal re-renders with the same lists)
    out["n_contrib"] = e.n_contrib.view(H, W).cpu().numpy()
    del e, params, img, hz
    torch.cuda.empty_cache()
    return out


def test_memory_holds_no_per_pair_state(large):
    """Peak device memory of the whole step: the five parameter-sized arrays
    (x, two EMAs, gradient, z . Gz: 7.1 GB at 6M) plus the records, the pair
    lists and the images; well under the 280 GB of the device."""
    f = large
    extra = f["peak"] - f["state_bytes"]
    print(f"\nlarge scene: peak {f['peak'] / 1e9:.2f} GB, parameter-sized arrays {f['state_bytes'] / 1e9:.2f} GB")
    assert f["peak"] < 24e9, f["peak"]
    assert extra < 8e9, extra


def test_sampled_pixels_match_oracle(large):
    f = large
    P = O.params64(f["sc"])
    rng = np.random.default_rng(8)
    xs = rng.integers(0, W, 256)
    ys = rng.integers(0, H, 256)
    with O.footprint_bins():  # the engine's default binning
        ref = O.render_pixels(P, DEG, f["cam"], xs, ys, outcomes=64)
    # each pixel equals one of the results the blend reaches when the decisions
    # FP32 may flip go either way
    img = f["img"][:, ys, xs].T
    ok, matched, _ = O.match_outcomes(ref, img, f["final_T"][ys, xs], img_tol=1e-5, flip_max=5e-6)
    print(f"\nlarge scene: {int((~ok).sum())} of {len(xs)} sampled pixels unresolved")
    assert (~ok).mean() <= 1e-4, int((~ok).sum())
    assert np.all(matched[ok])
    nc = f["n_contrib"][ys, xs]
    assert np.all(((nc >= ref["n_contrib_lo"]) & (nc <= ref["n_contrib_hi"]))[ok])


def test_sampled_gaussians_match_oracle(large):
    f = large
    P = O.params64(f["sc"])
    # samples chosen by the oracle's projection: visible, among the nearest fifth
    pr = O.project(P, DEG, f["cam"])
    cand = np.nonzero(pr["radius"] > 0)[0]
    cand = cand[np.argsort(pr["depth"][cand])[: max(64, len(cand) // 5)]]
    rng = np.random.default_rng(9)
    smp = rng.choice(cand, 64, replace=False)
    ref = O.backward_sampled(P, DEG, [f["cam"]], f["target"].astype(np.float64), smp, seed=42, t=f["t"], nu=1)
    # every sample is compared, with the oracle's allowances for flips of its own
    # decisions and residual signs (see the benchmark-size test)
    g_gpu, h_gpu = f["grad"][:, smp].T, f["hz"][:, smp].T
    g_ref, h_ref = ref["grad"], ref["hz"]
    g_mass, g_allow, g_round = ref["grad_mass"], ref["grad_allow"], ref["grad_round"]
    h_allow = ref["hz_sens"] + ref["hz_allow"]
    for name, sl in GROUPS.items():
        gs = np.abs(g_ref[:, sl]).max()
        hs = np.abs(h_ref[:, sl]).max()
        g_err = np.abs(g_gpu[:, sl] - g_ref[:, sl])
        assert np.all(g_err <= 1e-4 * gs + g_allow[:, sl]), name
        assert np.all(g_err <= 1e-4 * g_mass[:, sl] + g_allow[:, sl] + g_round[:, sl]), name
        assert np.all(np.abs(h_gpu[:, sl] - h_ref[:, sl]) <= 1e-3 * hs + h_allow[:, sl]), name
