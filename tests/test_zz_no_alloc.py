"""pot3d_residual_noalloc, the residual for callers that cannot allocate
device memory during the call (device memory owned by another allocator, a
fixed memory budget, or code where an allocation would synchronise the
device), against pot3d_residual (which uses memory its plan allocated).
Collected last on purpose, so that a run that stops at the first failure
has run every other test before this one."""
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


@pytest.mark.parametrize("shape,solved", [((11, 19, 45), False), ((13, 21, 37), True)])
def test_noalloc_residual_matches_residual(p3, shape, solved):
    nr, nt, np_ = shape
    plan = p3.Plan(*shape, ratio=1.04)
    br = torch.from_numpy(syn.bipole_br(nt, np_, seed=7, n_bipoles=20)).cuda()
    phi = torch.from_numpy(syn.random_field(shape, seed=8)).cuda()
    if solved:
        plan.solve(br, 1e-11, phi)
    ref = plan.residual(br, phi)
    # two calls in a row: the second reuses the scratch the first left behind
    first = plan.residual_noalloc(br, phi)
    second = plan.residual_noalloc(br, phi)
    for v in (first, second):
        assert abs(v - ref) <= 1e-12 * ref, (v, ref)
    plan.close()


def test_noalloc_allocates_nothing_and_follows_the_stream(p3):
    """A warm call leaves the device's free memory unchanged, and on a
    non-default torch stream it gives the same value as pot3d_residual."""
    shape = (12, 17, 40)
    plan = p3.Plan(*shape, ratio=1.03)
    br = torch.from_numpy(syn.bipole_br(17, 40, seed=9, n_bipoles=10)).cuda()
    phi = torch.from_numpy(syn.random_field(shape, seed=10)).cuda()
    ref = plan.residual(br, phi)
    plan.residual_noalloc(br, phi)  # warm: the kernels' module is loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    v = plan.residual_noalloc(br, phi)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert abs(v - ref) <= 1e-12 * ref
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        vals = [plan.residual_noalloc(br, phi) for _ in range(2)]
    s.synchronize()
    for w in vals:
        assert abs(w - ref) <= 1e-12 * ref, (w, ref)
    plan.close()


def test_noalloc_rejects_host_arrays(p3):
    plan = p3.Plan(4, 5, 8)
    br = np.zeros((5, 8))
    phi = np.zeros((4, 5, 8))
    rc, _ = plan.residual_noalloc(br, phi, check=False)
    assert rc == p3.POT3D_ERR_INVALID_ARG
    plan.close()
