"""The tensor-core kernels' bounded waits (every mbarrier wait gives up after a time limit, records
an error code and lets the kernel leave): otlm_check_wait_expiry runs a small GEMM whose first CTA
never issues its first copies, with a 20 ms limit, on the one-SM and the two-SM kernel.  The call
returns OTLM_ETIMEOUT with the recorded code, and the device stays usable: a solve afterwards
still matches the FP64 oracle.  No fault and no hang is involved: only the waits run out."""
import numpy as np
import pytest

import oracle
import spectra

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_04609_gb300 import otlm as api  # noqa: E402


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


@pytest.mark.parametrize("two_sm", [False, True])
def test_expired_waits_are_reported_and_the_device_stays_usable(two_sm):
    rc, code = api.check_wait_expiry(two_sm)
    assert rc == api.OTLM_ETIMEOUT, (rc, code)
    assert code in (1, 2, 3), code
    # a tensor-core solve right after (both kernels: 130 problems use the two-SM apply)
    d = spectra.batch(38, 130, 160, 8, 3)
    x, D, y = (torch.tensor(d[key], device="cuda") for key in ("x", "D", "y"))
    w0 = torch.tensor(spectra.initial_weights(d["y"], d["D"]), dtype=torch.float32, device="cuda")
    args = (1e-2, 1.0, 1e-3, "l2", "l2sq")
    r = api.solve(x, D, y, *args[:3], args[3], args[4], w0, max_iter=12, precision="bf16tc", poll_every=4)
    torch.cuda.synchronize()
    C = spectra.squared_cost(d["x"].astype(np.float64))
    D64 = d["D"].astype(np.float64)
    for p in (0, 129):
        y64 = d["y"][p].astype(np.float64)
        o = oracle.solve_log(C, D64, y64, *args, spectra.initial_weights(y64, D64), 12)
        assert rel_l1(r.w[p].cpu().numpy(), o["w"]) <= 1e-5
        assert rel_l1(r.t[p].cpu().numpy(), o["t"]) <= 1e-5
