"""The bounded device-side waits of the tensor-core gridding, exercised
without a fault: mmsar_plan_set_wait_test makes one MMA thread per CTA wait on
a barrier that nothing completes.  The wait runs out (about half a second),
the CTA's other roles stop, the image is void and the error word says
MMSAR_ERR_DEVICE_TIMEOUT; the context stays usable and the next image (test
switch off) matches the oracle."""
import time

import numpy as np
import pytest

import synth
from oracle import rma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_expired_wait_reports_timeout_and_the_context_survives(dev):
    from paper_2305_02064_gb300 import MmsarError, Plan
    scan = synth.custom(nx_pos=12, ny_pos=10, nk=96, layout="3x4", nx=32, ny=24, nz=12, seed=4, snr_db=30)
    plan = Plan.for_scan(scan)
    plan.set_tiles(2, 4, 0, 5)
    ws = plan.new_workspace(dev)
    vol = torch.zeros(plan.volume_shape, dtype=torch.complex64, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    args = (t(scan.echo), t(np.asarray(scan.pos, np.float64)), t(np.asarray(scan.tx, np.float64)),
            t(np.asarray(scan.rx, np.float64)))

    plan.set_wait_test(True)
    t0 = time.time()
    plan.image(ws, *args, vol)
    with pytest.raises(MmsarError, match="DEVICE_TIMEOUT"):
        plan.poll_error(ws)
    assert time.time() - t0 < 30.0   # every wait is bounded

    plan.set_wait_test(False)
    plan.image(ws, *args, vol)
    plan.poll_error(ws)   # the workspace header is reset per image
    got = vol.cpu().numpy()
    assert rma.nmse(got, rma.rma_exact(rma.setup_from(scan))) <= 2e-5

