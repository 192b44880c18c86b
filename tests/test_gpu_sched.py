"""Scheduler on the GPU: the doubles step recorded on a tamm_sched and run by dependency level (the
split-precision contractions of a level as one grouped launch) equals the step run operation by operation,
bit for bit, in split precision and FP64; it replays from a CUDA graph; and it matches the oracle."""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu


def test_scheduled_doubles_step(gpu_lib):
    import torch

    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles()
    stream = torch.cuda.Stream(0)
    ctx = gpu_lib.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        gsp, gt = gw.build(ctx, w)
        run = gw.Runner(ctx, w, gsp, gt)
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        for prec in ("ozaki_bf16", "f64"):
            run.run(prec, 0, energy_out=e.data_ptr())
            ctx.sync()
            ref = {k: gt[k].download() for k in ("R", "W")}
            e_ref = float(e.item())
            gt["R"].data.fill_(3.0)
            gt["W"].data.fill_(3.0)
            e.zero_()
            sch = run.scheduled(prec, 0, energy_out=e.data_ptr())
            assert sch.levels() == [0, 0, 1, 2, 0, 3, 4, 0]
            sch.execute()
            ctx.sync()
            for k in ("R", "W"):
                assert np.array_equal(gt[k].download(), ref[k]), (prec, k)
            assert float(e.item()) == e_ref
        sch = run.scheduled("ozaki_bf16", 0, energy_out=e.data_ptr())
        sch.execute()
        ctx.sync()
        eager = gt["R"].download()
        gt["R"].data.zero_()
        with ctx.capture() as cap:
            sch.execute()
        cap.graph.launch()
        ctx.sync()
        assert np.array_equal(gt["R"].download(), eager)
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    assert rel_err(gpu_to_oracle_layout(gt["R"], ot["R"]), ot["R"].data) <= 1e-10


RESIDUAL_OUT = ("R1", "R2", "Woooo", "Wvvvv", "Wovvo", "Fvv", "Foo", "Fov")


@pytest.mark.parametrize("shape", [(8, 24, 2, 4), (10, 34, 4, 7)], ids=["even", "ragged"])
def test_scheduled_ccsd_residual(gpu_lib, shape):
    """The full CCSD residual (55 operations, 11 dependency levels): scheduled = operation by operation
    bit for bit, replayed from one CUDA graph, and equal to the oracle running the recipe step by step
    (FP64 <= 1e-12, split precision <= 1e-10) for the T1 and T2 residuals, the intermediates and the
    energies."""
    import torch

    from paper_2201_01257_gb300 import workload as gw

    w = wl.ccsd_residual(*shape)
    _, ot = O.build_workload(w)
    oe = O.run_workload(w, ot)
    names = [s.name for s in w.steps if isinstance(s, wl.EnergySpec)]
    stream = torch.cuda.Stream(0)
    ctx = gpu_lib.Context(0, stream=stream)
    with torch.cuda.stream(stream):
        gsp, gt = gw.build(ctx, w)
        run = gw.Runner(ctx, w, gsp, gt)
        e = torch.zeros(len(names), dtype=torch.float64, device="cuda")
        for prec, tol in (("f64", 1e-12), ("ozaki_bf16", 1e-10)):
            run.run(prec, 0, energy_out=e.data_ptr())
            ctx.sync()
            ref = {k: gt[k].download() for k in RESIDUAL_OUT}
            e_seq = e.cpu().numpy().copy()
            for k in RESIDUAL_OUT:
                err = rel_err(gpu_to_oracle_layout(gt[k], ot[k]), ot[k].data)
                assert err <= tol, (prec, k, err)
            for n, x in zip(names, e_seq):
                assert abs(x - oe[n]) <= tol * abs(oe[n]), (prec, n, x, oe[n])
            for k in RESIDUAL_OUT:
                gt[k].data.fill_(7.0)
            e.zero_()
            sch = run.scheduled(prec, 0, energy_out=e.data_ptr())
            lev = sch.levels()
            assert len(lev) == len(w.steps) == 55 and max(lev) + 1 == 11
            sch.execute()
            ctx.sync()
            for k in RESIDUAL_OUT:
                assert np.array_equal(gt[k].download(), ref[k]), (prec, k)
            assert np.array_equal(e.cpu().numpy(), e_seq)
            # the scheduled residual captured once and replayed from a graph
            for k in RESIDUAL_OUT:
                gt[k].data.fill_(-1.0)
            with ctx.capture() as cap:
                sch.execute()
            cap.graph.launch()
            ctx.sync()
            for k in RESIDUAL_OUT:
                assert np.array_equal(gt[k].download(), ref[k]), (prec, "graph", k)
            # keep this graph alive across the next capture: its destruction is deferred to the end of
            # that capture, which must still succeed
            prev = cap.graph
        with ctx.capture() as cap2:
            prev.destroy()
            sch.execute()
        cap2.graph.launch()
        ctx.sync()
        cap2.graph.destroy()
