"""Host-side logic of bench.py that needs no GPU: the max-over-ranks timing of
a multi-replica run (two gloo ranks on the CPU), the algorithmic byte count
per PCG iteration, the kernel-source key of the recorded ncu traffic and its
scaling to another workload."""
import os
import socket

import numpy as np
import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, values, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        out[rank] = bench.max_over_ranks(values[rank], ws, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    values = [3.25, 7.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 7.5


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks(1.5, 1, "cpu") == 1.5


def test_algorithmic_bytes_count():
    """Two levels (3x3 fine, 6x6 coarsest), FP64 and FP32 V-cycles, 1 and 6
    load cases, against the terms written out by hand."""
    lv = [dict(n_rows=10, block=3, nnzb=40, nnzb_P=12), dict(n_rows=2, block=6, nnzb=4, nnzb_P=0)]
    n0, N0, N1 = 10, 30, 12
    A0 = 40 * (9 * 8 + 4) + 4 * (n0 + 1)
    for prec, w, wv in ((0, 8, 8), (1, 4, 4)):
        mat = A0 + N1 * N1 * 8
        Ab = 40 * (9 * w + 4) + 4 * 11
        Pb = 12 * (18 * w + 4) + 4 * 11
        Rb = 12 * (18 * w + 4) + 4 * 3
        Mb = 10 * 9 * wv
        mat += 2 * Mb + 2 * Ab + Pb + Rb
        vec = N0 * 8 * 2 + N0 * 8 * 11 + 2 * N1 * wv + 11 * N0 * wv + 2 * N1 * wv
        if prec:
            vec += N0 * 12 * 2
        for nr in (1, 6):
            assert bench.algorithmic_bytes_per_iteration(lv, prec, nr) == mat + nr * vec


def test_algorithmic_bytes_gauss_seidel_reads_each_operator_once_more():
    """The hybrid Gauss-Seidel V-cycle's pre-smoothing is a full sweep: A_l
    of every level but the coarsest is read once more than in the Jacobi
    V-cycle (whose pre-smoothing only applies M^+), plus the sweep's x."""
    lv = [dict(n_rows=10, block=3, nnzb=40, nnzb_P=12), dict(n_rows=4, block=6, nnzb=10, nnzb_P=3),
          dict(n_rows=1, block=6, nnzb=1, nnzb_P=0)]
    for prec, w, wv in ((0, 8, 8), (1, 4, 4)):
        jac = bench.algorithmic_bytes_per_iteration(lv, prec)
        gs = bench.algorithmic_bytes_per_iteration(lv, prec, gs=True)
        A0 = 40 * (9 * w + 4) + 4 * 11
        A1 = 10 * (36 * w + 4) + 4 * 5
        assert gs - jac == A0 + A1 + 30 * wv + 24 * wv


def test_algorithmic_bytes_bf16_below_level_0():
    """BF16 storage below level 0: level 0's A, P, R count 4 bytes per value,
    level 1's A, P, R 2 bytes; vectors as in the FP32 V-cycle."""
    lv = [dict(n_rows=10, block=3, nnzb=40, nnzb_P=12), dict(n_rows=4, block=6, nnzb=10, nnzb_P=3),
          dict(n_rows=1, block=6, nnzb=1, nnzb_P=0)]
    b1 = bench.algorithmic_bytes_per_iteration(lv, 1)
    b3 = bench.algorithmic_bytes_per_iteration(lv, 3)
    # only level 1's operators change: A_1 twice (residual, smoothing), P_1 and R_1 once
    saved = 2 * 10 * 36 * 2 + 3 * 36 * 2 + 3 * 36 * 2
    assert b1 - b3 == saved


def test_kernel_source_key_finds_every_named_kernel():
    src = os.path.join(os.path.dirname(bench.__file__), "paper_2011_13325_gb300", "csrc", "pcg.cu")
    a = bench.kernel_source_sha1(src, "pcg_spmv_dot_sell_df_kernel")
    b = bench.kernel_source_sha1(src, "pcg_spmv_dot_sell_kernel")
    assert a != b


def test_operator_complexity_counts_entries():
    lv = [dict(n_rows=100, block=3, nnzb=1000), dict(n_rows=10, block=6, nnzb=50)]
    oc = bench.operator_complexity(lv)
    assert oc["entries"] == round((9000 + 50 * 36) / 9000, 3)
    assert oc["blocks"] == 1.05 and oc["vertex"] == 1.1


def test_kernel_source_key_tracks_the_kernel(tmp_path):
    src = os.path.join(os.path.dirname(bench.__file__), "paper_2011_13325_gb300", "csrc",
                       "bsr_kernels.cu")
    text = open(src).read()
    h = bench.kernel_source_sha1(src, "sell_kernel")
    assert h == bench.kernel_source_sha1(src, "sell_kernel")
    # a change elsewhere keeps the key, a change inside the kernel does not
    other = tmp_path / "a.cu"
    other.write_text(text.replace("namespace amg {", "namespace amg {\n// note", 1))
    assert bench.kernel_source_sha1(str(other), "sell_kernel") == h
    i = text.index(" sell_kernel(int n_rows")
    j = text.index("if (row >= n_rows) return;", i)
    changed = tmp_path / "b.cu"
    changed.write_text(text[:j] + "if (row >= n_rows + 0) return;" + text[j + len("if (row >= n_rows) return;"):])
    assert bench.kernel_source_sha1(str(changed), "sell_kernel") != h


def test_traffic_is_scaled_to_the_workload():
    """The recorded capture applies unchanged only to the workload it was
    taken on; another workload gets it scaled by the algorithmic bytes."""
    rec = {"workload": "cube64", "bytes_per_launch": 296559360,
           "algorithmic_bytes_per_launch": 300257852}
    t, kind = bench.scaled_traffic(rec, 300257852)
    assert t == 296559360 and "capture (cube64)" in kind
    # a launch with twice the algorithmic bytes: twice the traffic
    t, kind = bench.scaled_traffic(rec, 2 * 300257852)
    assert t == 2 * 296559360 and "scaled" in kind
    # the committed record names its workload, and its traffic is close to
    # (not far above) the algorithmic bytes of that launch
    committed = bench.traffic_record("pcg_spmv_dot_sell_df_kernel<3>")
    if committed is not None:
        assert committed["algorithmic_bytes_per_launch"] > committed["bytes_per_launch"] * 0.9
    assert bench.scaled_traffic(None, 1) == (None, None)


def test_batch_stage_roofline_bytes():
    """One system, two levels: the residual and restriction stages of level 0
    and the FP64 CG product, against the byte counts written out."""
    lv = [[dict(n_rows=10, block=3, nnzb=40, nnzb_P=12), dict(n_rows=2, block=6, nnzb=4, nnzb_P=0)]]
    tuned = ["iteration: level 0 t = b - A x (low precision) 3x3: 1 systems, 5 blocks, 32 lanes/row, "
             "4 warps/block, 2.0 us",
             "iteration: level 0 b_c = R t (low precision) 6x3: 1 systems, 5 blocks, SELL-32 thread/row, "
             "2 slices/block, 1.0 us",
             "iteration: q = A_0 p 3x3: 1 systems, 5 blocks, SELL-32 thread/row, 2 slices/block, 4.0 us"]
    out = {r["stage"].split(" (")[0]: r for r in bench.batch_stage_roofline(lv, tuned, 1, 1000.0, nr=6)}
    resid = 40 * (9 * 4 + 4) + 4 * 11 + 3 * 30 * 6 * 4
    restr = 12 * (18 * 4 + 4) + 4 * 3 + (30 + 12) * 6 * 4
    cg = 40 * (9 * 8 + 4) + 4 * 11 + 2 * 30 * 6 * 8
    assert out["level 0 t = b - A x"]["mbytes"] == round(resid / 1e6, 1)
    assert abs(out["level 0 t = b - A x"]["gbs"] - round(resid / 2e-6 / 1e9, 1)) < 1e-9
    assert abs(out["level 0 b_c = R t"]["gbs"] - round(restr / 1e-6 / 1e9, 1)) < 1e-9
    assert abs(out["q = A_0 p"]["gbs"] - round(cg / 4e-6 / 1e9, 1)) < 1e-9


def test_clock_sampler_parses_nvidia_smi_lines():
    """Median SM clock, maximum, and the throttle reasons that were active
    in any sample, from nvidia-smi's csv lines (the fields ClockSampler asks
    for)."""
    lines = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])

    class Proc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            return lines, ""

    s = bench.ClockSampler(0)
    s.proc = Proc()
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.proc = None
    assert s.stop() is None


def test_batch_oracle_uses_its_own_iteration_counts():
    """The batched CPU legs (cpu_baseline and the reference arm): the C
    oracle rebuilt from downloaded prolongations (here the oracle's own)
    solves every load case to rtol with the numpy oracle's iteration counts
    (never the GPU's), and the bounded sample scales per dof-iteration to
    every load case at those counts."""
    from oracle import hierarchy, solve
    from workloads import configs, make_problem
    probs = [make_problem(shape, seed=seed, h=1.0 / 32, forces=configs.SIX_LOADS)
             for shape, seed in (((6, 5, 5), 2), ((5, 6, 7), 3))]
    P_lists, want = [], []
    for p in probs:
        H = hierarchy.setup(p, hierarchy.SetupParams(coarse_max=4))
        P_lists.append([(P.n_rows, P.n_cols, P.rowptr.astype(np.int32), P.colidx.astype(np.int32),
                         P.vals) for P in H.P])
        want += [solve.pcg(H, p.b[j], rtol=1e-8)[1] for j in range(p.b.shape[0])]
    ob = bench.OracleBatch(probs, P_lists, 1e-8)
    ms, its = ob.solve_all()
    assert ms > 0 and len(its) == 6 * len(probs)
    assert all(abs(a - b) <= 1 for a, b in zip(its, want)), (its, want)
    v, sample = ob.sample(budget_s=0.05)
    assert v > 0 and "own iteration counts" in sample


def test_oracle_leg_on_cpu():
    """The bench's CPU oracle leg on a small hierarchy (the oracle's own
    prolongations): the all-thread solve reaches rtol with the numpy
    oracle's iteration count, the one-thread sample scales to it, and the
    energy error of the numpy oracle's 1e-8 solution is small."""
    import types
    from oracle import hierarchy, solve
    from workloads import configs
    p = configs.square32()
    H = hierarchy.setup(p)
    P_list = [(P.n_rows, P.n_cols, P.rowptr.astype(np.int32), P.colidx.astype(np.int32), P.vals)
              for P in H.P]
    u, it, _ = solve.pcg(H, p.b[0], rtol=1e-8)
    args = types.SimpleNamespace(rtol=1e-8)
    cpu, acc = bench.oracle_leg(p, P_list, None, args, u, {"same": u}, it, single_budget_s=0.2)
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and abs(cpu["iters"] - it) <= 1
    assert cpu["value"] > 0 and cpu["single_thread"]["cores"] == 1
    assert acc["energy_error"] <= 1e-6 and acc["variants"]["same"] == acc["energy_error"]
    assert acc["oracle_1e8"] <= 1e-6


def test_oracle_leg_follows_the_gauss_seidel_smoother():
    """With --smoother gs the CPU legs run the oracle with the hybrid
    Gauss-Seidel smoother: the numpy oracle's GS iteration count, not the
    block-l1 Jacobi one."""
    import types
    from oracle import hierarchy, solve
    from workloads import make_problem
    p = make_problem((9, 7, 8), seed=3, jump_boxes=6, nu_range=(0.25, 0.45))
    H = hierarchy.setup(p, hierarchy.SetupParams(coarse_max=6))
    P_list = [(P.n_rows, P.n_cols, P.rowptr.astype(np.int32), P.colidx.astype(np.int32), P.vals)
              for P in H.P]
    Hg = solve.prepare(H.A[0], H.P, smoother="hybrid_gs")
    u, it_gs, _ = solve.pcg(Hg, p.b[0], rtol=1e-8)
    it_j = solve.pcg(H, p.b[0], rtol=1e-8)[1]
    assert it_gs != it_j
    args = types.SimpleNamespace(rtol=1e-8, smoother="gs")
    cpu, _ = bench.oracle_leg(p, P_list, None, args, u, {}, it_gs, skip_accuracy=True,
                              single_budget_s=0.05)
    assert abs(cpu["iters"] - it_gs) <= 1 and "hybrid_gs" in cpu["sample"]
    assert bench.oracle_smoother(types.SimpleNamespace(smoother="l1")) == "l1_jacobi"


@pytest.mark.parametrize("smoother", ["l1", "gs"])
def test_reference_arm_line_on_cpu(monkeypatch, capsys, smoother):
    """bench.py --impl reference on the 2D workload, with the library's
    setup replaced by a stand-in that hands over the oracle's prolongations
    (the setup needs a GPU): one JSON line with the contract's keys, the
    oracle's smoother named, the value equal to cpu_baseline and e2e."""
    import json
    import types
    from oracle import hierarchy
    from paper_2011_13325_gb300 import amg

    class FakeContext:
        def __init__(self, device):
            self.P = None

        def setup(self, problem, prec, **kw):
            H = hierarchy.setup(problem, hierarchy.SetupParams(
                coarse_max=kw.get("coarse_max", 0) or hierarchy.SetupParams().coarse_max))
            self.P = H.P
            self.n_levels = H.n_levels

        def download_prolongation(self, l):
            P = self.P[l]
            return (P.n_rows, P.n_cols, P.rowptr.astype(np.int32), P.colidx.astype(np.int32), P.vals)

        def close(self):
            pass

    monkeypatch.setattr(amg, "Context", FakeContext)
    args = types.SimpleNamespace(workload="square32", steps=2, warmup=3, rtol=1e-8, smoother=smoother)
    bench.run_reference(args, 1, 0, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is False
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    want = {"l1": "block-l1 Jacobi", "gs": "block-l1 hybrid Gauss-Seidel (colour classes)"}[smoother]
    assert line["config"]["workload"] == "square32" and line["config"]["smoother"] == want
    assert ("hybrid_gs" in line["cpu_baseline"]["sample"]) == (smoother == "gs")
