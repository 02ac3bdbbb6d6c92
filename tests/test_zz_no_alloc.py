"""pot3d_residual_noalloc, the residual for callers that cannot allocate
device memory during the call, against pot3d_residual (which uses memory
its plan allocated).  Collected last on purpose."""
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
    first = plan.residual_noalloc(br, phi)
    second = plan.residual_noalloc(br, phi)
    for v in (first, second):
        assert abs(v - ref) <= 1e-12 * ref, (v, ref)
    plan.close()


def test_noalloc_rejects_host_arrays(p3):
    plan = p3.Plan(4, 5, 8)
    br = np.zeros((5, 8))
    phi = np.zeros((4, 5, 8))
    rc, _ = plan.residual_noalloc(br, phi, check=False)
    assert rc == p3.POT3D_ERR_INVALID_ARG
    plan.close()
