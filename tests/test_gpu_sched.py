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
