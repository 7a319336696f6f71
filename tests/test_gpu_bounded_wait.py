"""The bounded device wait runs out without faulting or hanging: a barrier
that nothing arrives at is polled a fixed number of times, the timeout status
comes back to the host, and the context stays usable (a solve afterwards is
correct)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_12742_gb300 import hines as H
from paper_1810_12742_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_reports_timeout():
    status, ns = H.check_bounded_wait(1000, arrive=False)
    assert status == H.HINES_ERR_TIMEOUT
    assert ns > 0
    print(f"1000 polls with nothing arriving: {ns / 1e3:.1f} us")
    status, _ = H.check_bounded_wait(1000, arrive=True)
    assert status == H.HINES_OK
    # the context is still usable
    pop = I.population("fp64_small", cells=np.arange(8))
    plan = H.Plan(pop["ncomp"], pop["parent"])
    x = torch.as_tensor(pop["b"]).cuda()
    H.solve(plan, torch.as_tensor(pop["d"]).cuda(), torch.as_tensor(pop["u"]).cuda(), x)
    ref = oracle.solve_batch(pop["ncomp"], pop["parent"], pop["d"], pop["u"], pop["b"])
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert plan.status() == 0
