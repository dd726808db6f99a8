"""amg_vcycle_static, the V-cycle entry point that allocates nothing (its
work vectors live in a fixed device array of the library).  It serves callers
that cannot allocate device memory while it runs: a framework whose caching
allocator already holds the free device memory, or code with a memory budget
fixed in advance.

Checked here: on two calls in a row (which share the array) it gives the
V-cycle of amg_vcycle and of the oracle (Algorithm tg applied recursively)
element by element, in all four V-cycle precisions; a call after the first
changes the free device memory by nothing; hierarchies whose work vectors do
not fit are rejected.  Collected last on purpose (the file name), so that a
run stopping at its first failure has run every other test before."""
import numpy as np
import pytest

from oracle import hierarchy, solve
from workloads import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# element-wise tolerance against the FP64 oracle V-cycle, per precision:
# FP64 as the other V-cycle parity tests; for FP32 / BF16 storage, the oracle
# V-cycle run with the operators rounded to FP32 / BF16 differs from the FP64
# one by at most 8e-8 / 5.3e-3 (max-norm relative, on these meshes); the
# bounds leave room for the FP32 vector arithmetic on top
ORACLE_TOL = {0: 1e-10, 1: 1e-5, 2: 2e-2, 3: 2e-2}

_H = {}


def _hier(shape, params):
    key = (shape, tuple(sorted(params.items())))
    if key not in _H:
        p = make_problem(shape, seed=1 if len(shape) == 2 else 2)
        _H[key] = (p, hierarchy.setup(p, hierarchy.SetupParams(**params)))
    return _H[key]


def _maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("shape,params", [((33, 33), {}), ((10, 10, 10), {"coarse_max": 8})])
def test_static_vcycle_matches_vcycle_twice(shape, params, prec):
    from paper_2011_13325_gb300 import amg
    p, H = _hier(shape, params)
    ctx = amg.Context(0)
    ctx.upload_hierarchy(H.A[0], H.P, prec)
    n = H.A[0].n_rows * H.A[0].br
    rng = np.random.default_rng(3)
    for call in range(2):   # two calls in a row share the device array
        r_h = rng.normal(size=n)
        r = torch.from_numpy(r_h).cuda()
        z_ref = torch.zeros_like(r)
        z = torch.full_like(r, float("nan"))
        ctx.vcycle(r, z_ref)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ctx.vcycle_static(r, z)
        torch.cuda.synchronize()
        if call == 1:      # the first call is the set-up; later ones allocate nothing
            assert torch.cuda.mem_get_info()[0] == free0
        zh, zr = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.isfinite(zh).all()
        # the same kernels on the same data: agrees with amg_vcycle to rounding
        assert _maxrel(zh, zr) <= 1e-12, (call, _maxrel(zh, zr))
        zo = solve.vcycle(H, r_h)
        assert _maxrel(zh, zo) <= ORACLE_TOL[prec], (call, prec, _maxrel(zh, zo))
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
