"""The Python binding's checks of array arguments, on the CPU: a vector handed
to libamg must be a CUDA tensor (device entries) or a numpy array / CPU
tensor (host entries), of the element type the C signature names, contiguous
and at least as long as the level it belongs to.  The library calls are
replaced by a fake that records what it receives, so no GPU is needed."""
import ctypes as C

import numpy as np
import pytest

from paper_2011_13325_gb300 import amg

torch = pytest.importorskip("torch")


class FakeCuda:
    """Stands in for a CUDA tensor (only the attributes the binding reads)."""

    def __init__(self, n, dtype="float64", index=0, contiguous=True):
        self._n, self.dtype, self._c = n, f"torch.{dtype}", contiguous
        self.is_cuda = True
        self.device = type("D", (), {"index": index, "__str__": lambda s: f"cuda:{index}"})()

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x1000


class FakeLib:
    """Level sizes of a two-level hierarchy: 10 block rows of 3x3, then 2 of
    6x6; every call records its arguments and returns AMG_OK."""

    def __init__(self, levels=((10, 3), (2, 6))):
        self.levels = levels
        self.calls = []

    def amg_level_info(self, h, level, n_rows, block, nnzb_a, nnzb_p, n_levels):
        if n_levels is not None:
            n_levels._obj.value = len(self.levels)
        if not self.levels:
            return amg.AMG_ERR_STATE
        if not 0 <= level < len(self.levels):
            return amg.AMG_ERR_ARG
        if n_rows is not None:
            n_rows._obj.value = self.levels[level][0]
        if block is not None:
            block._obj.value = self.levels[level][1]
        return amg.AMG_OK

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            return amg.AMG_OK
        return call


@pytest.fixture
def ctx(monkeypatch):
    fake = FakeLib()
    monkeypatch.setattr(amg, "lib", lambda: fake)
    c = object.__new__(amg.Context)
    c.h = C.c_void_p(1)
    c.device = 0
    try:
        yield c, fake
    finally:
        c.h = C.c_void_p()   # never hand the fake handle to the real library


def test_device_vectors_pass_when_right(ctx):
    c, fake = ctx
    c.spmv(0, FakeCuda(30), FakeCuda(30))
    c.restrict(0, FakeCuda(30), FakeCuda(12))
    c.prolong_add(0, FakeCuda(12), FakeCuda(30))
    c.coarse_solve(FakeCuda(12), FakeCuda(12))
    c.vcycle(FakeCuda(60), FakeCuda(60), nrhs=2)
    c.smooth(1, FakeCuda(12), None, FakeCuda(12))
    assert [n for n, _ in fake.calls] == ["amg_spmv", "amg_restrict", "amg_prolong_add",
                                          "amg_coarse_solve", "amg_vcycle", "amg_smooth"]
    assert fake.calls[-1][1][3] is None          # optional x_in passes as NULL


@pytest.mark.parametrize("bad,err", [
    (lambda: FakeCuda(29), ValueError),                      # shorter than level 0
    (lambda: FakeCuda(30, dtype="float32"), TypeError),      # wrong element type
    (lambda: FakeCuda(30, contiguous=False), ValueError),    # strided view
    (lambda: FakeCuda(30, index=1), ValueError),             # another GPU
    (lambda: np.zeros(30), TypeError),                       # host array to a device entry
    (lambda: torch.zeros(30, dtype=torch.float64), TypeError),  # CPU tensor likewise
])
def test_device_vectors_rejected(ctx, bad, err):
    c, fake = ctx
    with pytest.raises(err):
        c.spmv(0, bad(), FakeCuda(30))
    with pytest.raises(err):
        c.pcg_solve(FakeCuda(30), bad())
    assert fake.calls == []


def test_coarse_level_lengths(ctx):
    c, _ = ctx
    with pytest.raises(ValueError):
        c.restrict(0, FakeCuda(30), FakeCuda(11))    # level-1 vector is 2 x 6
    with pytest.raises(ValueError):
        c.vcycle(FakeCuda(30), FakeCuda(30), nrhs=2)  # two load cases need 60


def test_host_entry(ctx):
    c, fake = ctx
    f = np.ones(30)
    u = torch.zeros(30, dtype=torch.float64)
    c.pcg_solve_host(f, u)
    name, args = fake.calls[-1]
    assert name == "amg_pcg_solve_host" and args[1] == f.ctypes.data and args[2] == u.data_ptr()
    with pytest.raises(TypeError):
        c.pcg_solve_host(FakeCuda(30), u)                     # device tensor to a host entry
    with pytest.raises(ValueError):
        c.pcg_solve_host(np.ones(60)[::2], u)                 # non-contiguous
    with pytest.raises(TypeError):
        c.pcg_solve_host(np.ones(30, dtype=np.float32), u)


def test_without_hierarchy_the_library_reports(monkeypatch):
    """No hierarchy: lengths are unknown, the call goes through and the
    library's own status (AMG_ERR_STATE) reaches the caller."""
    fake = FakeLib(levels=())
    fake.amg_spmv = lambda *a: amg.AMG_ERR_STATE
    fake.amg_last_error = lambda h: b"no hierarchy"
    monkeypatch.setattr(amg, "lib", lambda: fake)
    c = object.__new__(amg.Context)
    c.h, c.device = C.c_void_p(1), 0
    try:
        with pytest.raises(amg.AmgError) as e:
            c.spmv(0, FakeCuda(4), FakeCuda(4))
        assert e.value.code == amg.AMG_ERR_STATE
    finally:
        c.h = C.c_void_p()   # never hand the fake handle to the real library


def test_learned_arrays(ctx):
    c, fake = ctx
    c.learned_features(np.zeros((10, 3)), FakeCuda(130, dtype="float32"), FakeCuda(10))
    c.learned_targets(T32=FakeCuda(90, dtype="float32"))
    with pytest.raises(TypeError):
        c.learned_targets(T32=FakeCuda(90))                   # FP64 where FP32 is named
    with pytest.raises(ValueError):
        c.learned_features(np.zeros((9, 3)), FakeCuda(130, dtype="float32"))
    with pytest.raises(ValueError):
        c.learned_features(np.zeros((10, 3)), FakeCuda(129, dtype="float32"))


def test_pointer_helper_plain():
    a = np.arange(5.0)
    assert amg._ptr(a, host=True, n=5) == a.ctypes.data
    assert amg._ptr(None) is None
    with pytest.raises(ValueError):
        amg._ptr(a, host=True, n=6)
    with pytest.raises(TypeError):
        amg._ptr([1.0, 2.0], host=True)


def test_learned_smoother_coords(ctx):
    c, fake = ctx
    net = type("N", (), {"h": C.c_void_p(2)})()
    c.set_learned_smoother(net, np.zeros((10, 3)))
    assert fake.calls[-1][0] == "amg_set_learned_smoother"
    with pytest.raises(ValueError):
        c.set_learned_smoother(net, np.zeros((9, 3)))


def test_batch_vectors(monkeypatch):
    """Stacked batch vectors: device entry wants CUDA tensors on the
    contexts' GPU, host entry numpy / CPU tensors, both the full stacked
    length that amg_batch_layout reports."""
    fake = FakeLib()

    def layout(h, s, off, n, total):
        for p, v in ((off, 0), (n, 30), (total, 180)):
            if p is not None:
                p._obj.value = v
        return amg.AMG_OK
    fake.amg_batch_layout = layout
    monkeypatch.setattr(amg, "lib", lambda: fake)
    b = object.__new__(amg.Batch)
    b.h = C.c_void_p(1)
    b.nrhs = 6
    b.contexts = [type("Cx", (), {"device": 0})()]
    try:
        _batch_checks(b, fake)
    finally:
        b.h = C.c_void_p()   # never hand the fake handle to the real library


def _batch_checks(b, fake):
    b.pcg_solve(FakeCuda(180), FakeCuda(180))
    assert fake.calls[-1][0] == "amg_batch_pcg_solve"
    b.pcg_solve_host(np.zeros(180), torch.zeros(180, dtype=torch.float64))
    assert fake.calls[-1][0] == "amg_batch_pcg_solve_host"
    with pytest.raises(ValueError):
        b.pcg_solve(FakeCuda(179), FakeCuda(180))
    with pytest.raises(TypeError):
        b.pcg_solve_host(FakeCuda(180), np.zeros(180))
    with pytest.raises(TypeError):
        b.pcg_solve(np.zeros(180), FakeCuda(180))
