"""Failure detection on the GPU without a fault: a bounded device-side wait
on a barrier that nothing completes gives up after its limit, the kernel
reports the TIMEOUT status the iteration kernels use, the host reads it,
and the context stays usable."""
import time

import numpy as np
import pytest

import pot3d_synth as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def p3():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_01126_gb300 import pot3d

    pot3d.load(build_if_missing=True)
    return pot3d


def test_bounded_wait_reports_timeout_and_context_survives(p3, oracle_mod):
    t = time.perf_counter()
    st, elapsed = p3.selftest_wait(0.2)
    wall = time.perf_counter() - t
    assert st == p3.POT3D_ERR_TIMEOUT
    assert 0.2 <= elapsed < 2.0 and wall < 10.0
    # the same context still solves correctly
    shape = (9, 8, 64)
    br = syn.bipole_br(8, 64, seed=3, n_bipoles=8)
    g = oracle_mod.Grid(*shape, ratio=1.1)
    ref, it_ref, _ = g.solve(br, 1e-12)
    plan = p3.Plan(*shape, ratio=1.1)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rc, it = plan.solve(torch.from_numpy(br).cuda(), 1e-12, phi)
    assert rc == 0 and abs(it - it_ref) <= 1
    x = phi.cpu().numpy()
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-9
    plan.close()
