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


def test_batch_arena_larger_than_device_is_oom_without_leak(p3):
    """A batch arena larger than the device fails with POT3D_ERR_OOM, leaves
    the device's free memory as it was, and the next batch works."""
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    with pytest.raises(p3.Pot3dError) as ei:
        p3.Batch(2 * total, max_slots=4)
    assert ei.value.code == p3.POT3D_ERR_OOM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (2 << 20), (free0, free1)
    pl = p3.Plan(9, 12, 30, ratio=1.02, precision="mixed")
    b = p3.Batch(1 << 28, max_slots=4)
    br = torch.from_numpy(syn.bipole_br(12, 30, seed=4, n_bipoles=6)).cuda()
    phi = torch.zeros(pl.shape, dtype=torch.float64, device="cuda")
    assert b.submit(pl, br, 1e-10, phi, 7)
    done = []
    for _ in range(1000):
        b.step(16)
        done += b.poll()
        if done:
            break
    assert done and done[0][0] == 7 and done[0][1] == 0 and done[0][4] <= 1e-10
    b.close()
    pl.close()


@pytest.mark.parametrize("opts", [{"chunk": 2}, {"chunk": 2, "time_kernels": 1}])
def test_host_progress_guard_reports_timeout(p3, oracle_mod, opts):
    """The host's guard against a solve whose device state stops advancing:
    with the polled snapshot frozen (a testing hook; nothing on the device
    is disturbed) the solve ends with POT3D_ERR_TIMEOUT instead of polling
    forever, and the same plan then solves correctly."""
    shape, ratio = (12, 16, 40), 1.05
    br = syn.bipole_br(16, 40, seed=5, n_bipoles=10)
    g = oracle_mod.Grid(*shape, ratio=ratio)
    ref, it_ref, _ = g.solve(br, 1e-12)
    assert it_ref > 10
    plan = p3.Plan(*shape, ratio=ratio, precision="fp64", **opts)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    brd = torch.from_numpy(br).cuda()
    plan.test_freeze_poll(True)
    rc, it = plan.solve(brd, 1e-12, phi, check=False)
    assert rc == p3.POT3D_ERR_TIMEOUT
    plan.test_freeze_poll(False)
    rc, it = plan.solve(brd, 1e-12, phi)
    assert rc == 0 and abs(it - it_ref) <= 1
    assert np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-9
    plan.close()


def test_probe_fp64_fma_rate(p3):
    """The in-library DFMA throughput probe (the FP64 roofline denominator)
    returns a rate of the order of the FP64 units' nominal peak (152 SMs x
    2 DFMA per clock at up to 2.07 GHz = 6.3e11 per second)."""
    rate, el = p3.probe_fp64_fma(0.2)
    assert el >= 0.2
    assert 1e11 < rate < 1.3e12, rate
