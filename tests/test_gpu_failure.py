"""Failure detection without a GPU fault.

Every kernel that waits on an asynchronous copy waits a bounded number of
tries, then raises GS_FLAG_TIMEOUT in the caller's status word and returns.
`gs_wait_check` runs that wait on an mbarrier that nothing completes (a flag
that nothing sets), so the limit always runs out: the status must report it,
the launch must finish, and the context must stay usable for the next step.
"""
import numpy as np
import pytest

from paper_2602_00395_gb300 import synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2602_00395_gb300 import gs3dtr as G
    from paper_2602_00395_gb300.engine import TRConfig, TRStep
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.gs_wait_check(1000, status)
    torch.cuda.synchronize()  # the kernel returned: no hang, no fault
    assert int(status.item()) == G.GS_FLAG_TIMEOUT
    # a clean status word stays clean when the wait is not reached
    status.zero_()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # the context still runs a full step, with a status word of its own
    sc = S.make_scene(500, 1, seed=1001, kind="cube", extent=1.0)
    cams = S.camera_ring(8, 96, 64, 1.0, seed=7)[:2]
    e = TRStep(sc.n, sc.sh_degree, 2, 96, 64, nu=1, cfg=TRConfig(l=1))
    e.set_cameras(cams)
    e.set_params(sc.params)
    e.set_target(S.smooth_target(2, 64, 96, seed=2001))
    e.ensure_capacity()
    e.step(1, 1e-3)
    torch.cuda.synchronize()
    assert e.read_status() == 0
    assert np.isfinite(e.x.cpu().numpy()).all()
