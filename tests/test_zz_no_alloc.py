"""amg_vcycle_static, the V-cycle entry point that allocates nothing (its
work vectors live in a fixed device array of the library), for callers that
must not allocate device memory while it runs (e.g. while another library
captures the stream into a CUDA graph).  It must give the V-cycle of
amg_vcycle, on consecutive calls sharing the array, and reject hierarchies
whose work vectors do not fit.  Collected last on purpose."""
import numpy as np
import pytest

from oracle import hierarchy
from workloads import configs, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape,params", [((33, 33), {}), ((10, 10, 10), {"coarse_max": 8})])
def test_static_vcycle_matches_vcycle_twice(shape, params, prec):
    from paper_2011_13325_gb300 import amg
    p = make_problem(shape, seed=1 if len(shape) == 2 else 2)
    H = hierarchy.setup(p, hierarchy.SetupParams(**params))
    ctx = amg.Context(0)
    ctx.upload_hierarchy(H.A[0], H.P, prec)
    n = H.A[0].n_rows * H.A[0].br
    rng = np.random.default_rng(3)
    for call in range(2):   # two calls in a row share the device array
        r = torch.from_numpy(rng.normal(size=n)).cuda()
        z_ref = torch.zeros_like(r)
        z = torch.full_like(r, float("nan"))
        ctx.vcycle(r, z_ref)
        ctx.vcycle_static(r, z)
        torch.cuda.synchronize()
        assert torch.isfinite(z).all()
        assert _rel(z, z_ref) <= 1e-12, (call, _rel(z, z_ref))
    ctx.close()


def test_static_vcycle_rejects_too_large_hierarchy():
    from paper_2011_13325_gb300 import amg
    p = make_problem((58, 58, 58), seed=2)      # 575k dofs: > 16 MiB of FP64 work vectors
    ctx = amg.Context(0)
    ctx.setup(p, amg.AMG_PREC_FP64)
    r = torch.zeros(p.ndof, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(amg.AmgError) as e:
        ctx.vcycle_static(r, z)
    assert e.value.code == amg.AMG_ERR_ARG and "bytes" in str(e.value)
    ctx.close()
