"""Shared scaling of the split-precision path (TAMM_OPT_OZAKI_SHARED_SCALE = 1): one exponent per output
row and column over every operand block that feeds it, so the exact accumulation chunks run across
block pairs.

* every doubles contraction (ladder, intermediate, oooo, ring with its output antisymmetriser, T1)
  against the oracle (<= 1e-10), on even and ragged tiles, with and without split summed ranges;
* tile policies, grid kinds and column panels give bitwise the same values under shared scaling;
* short summed ranges really share chunks: fewer accumulator drains show as the same values with
  one chunk length that spans block pairs (checked through the oracle);
* the autotuner reports its scaling choice and slices = 0 then reproduces it;
* the (T) correction with shared scaling against the oracle (<= 1e-10).
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu


def _run(tg, w, shared=1, split=1, policy=1, persistent=0, panels=1):
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    for opt, val in ((tg.TAMM_OPT_OZAKI_SHARED_SCALE, shared), (tg.TAMM_OPT_OZAKI_SPLIT_K, split),
                     (tg.TAMM_OPT_OZAKI_TILE_POLICY, policy), (tg.TAMM_OPT_OZAKI_PERSISTENT, persistent),
                     (tg.TAMM_OPT_OZAKI_PANELS, panels)):
        ctx.set_option(opt, val)
    gsp, gt = gw.build(ctx, w)
    gw.Runner(ctx, w, gsp, gt).run("ozaki_bf16", 0)
    ctx.sync()
    return ctx, gt


@pytest.mark.parametrize("shape", [(8, 24, 2, 4), (10, 34, 4, 7), (16, 64, 8, 16)],
                         ids=["even", "ragged", "split"])
def test_shared_scale_doubles_match_oracle(gpu_lib, shape):
    w = wl.small_doubles(*shape)
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    for split in (0, 1):
        _, gt = _run(gpu_lib, w, shared=1, split=split)
        for k in ("R", "W"):
            err = rel_err(gpu_to_oracle_layout(gt[k], ot[k]), ot[k].data)
            print(f"{shape} split={split} {k}: {err:.2e}")
            assert err <= 1e-10, (shape, split, k, err)


def test_shared_scale_each_term(gpu_lib):
    # each contraction alone, from a zeroed output, against the oracle
    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles(12, 36, 3, 5)
    _, ot = O.build_workload(w)
    ctx = gpu_lib.Context(0)
    ctx.set_option(gpu_lib.TAMM_OPT_OZAKI_SHARED_SCALE, 1)
    gsp, gt = gw.build(ctx, w)
    run = gw.Runner(ctx, w, gsp, gt)
    run.run("f64")  # W holds W0 + V_oovv T for the oooo term, on both sides
    O.run_workload(w, ot)
    W_ref = ot["W"].data.copy()
    for st in w.steps:
        if not isinstance(st, wl.ContractSpec) or st.c != "R":
            continue
        gt["R"].data.zero_()
        run.run("ozaki_bf16", 0, steps=[st])
        ctx.sync()
        R = O.Tensor(ot["R"].modes, 2)
        ot_step = dict(ot)
        ot_step["R"] = R
        ot_step["W"].data[:] = W_ref
        O.run_step(w, ot_step, st)
        err = rel_err(gpu_to_oracle_layout(gt["R"], R), R.data)
        print(st.name, f"{err:.2e}")
        assert err <= 1e-10, (st.name, err)


def test_shared_scale_invariant_to_work_split(gpu_lib):
    w = wl.small_doubles(16, 40, 8, 10)
    outs = []
    for policy in (0, 1, 2, 3):
        for persistent in (0, 1):
            for panels in (0, 1):
                _, gt = _run(gpu_lib, w, policy=policy, persistent=persistent, panels=panels)
                outs.append({k: gt[k].download() for k in ("R", "W")})
    for k in ("R", "W"):
        for p in range(1, len(outs)):
            assert np.array_equal(outs[p][k], outs[0][k]), (k, p)


def test_autotune_reports_and_reuses_scaling(gpu_lib):
    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles(12, 36, 3, 5)
    ctx = gpu_lib.Context(0)
    gsp, gt = gw.build(ctx, w)
    st = next(s for s in w.steps if s.name == "t1")
    tuned = gw.Runner(ctx, w, gsp, gt).autotune(1e-10, steps=[st])["t1"]
    assert tuned["shared_scale"] in (0, 1) and tuned["fused_a"] in (0, 1)
    assert not (tuned["shared_scale"] and tuned["fused_a"])
    R = gt["R"]
    ctx.contract(1.0, R, "abij", 0.0, gt["V_vvvo"], "abej", gt["t1"], "ei", "ozaki_bf16", 0)
    a = R.download()
    for opt, val in ((gpu_lib.TAMM_OPT_OZAKI_SHARED_SCALE, tuned["shared_scale"]),
                     (gpu_lib.TAMM_OPT_OZAKI_FUSED_A, tuned["fused_a"]),
                     (gpu_lib.TAMM_OPT_OZAKI_CHUNK_K, tuned["chunk_k"]),
                     (gpu_lib.TAMM_OPT_OZAKI_TILE_POLICY, tuned["tile_policy"]),
                     (gpu_lib.TAMM_OPT_OZAKI_PERSISTENT, tuned["persistent"])):
        ctx.set_option(opt, val)
    ctx.contract(1.0, R, "abij", 0.0, gt["V_vvvo"], "abej", gt["t1"], "ei", "ozaki_bf16", tuned["slices"])
    assert np.array_equal(R.download(), a)


def test_triples_shared_scale_matches_oracle(gpu_lib):
    import torch

    from paper_2201_01257_gb300 import workload as gw

    w = wl.triples(16, 64, 4, 16)
    ctx = gpu_lib.Context(0)
    ctx.set_option(gpu_lib.TAMM_OPT_OZAKI_SHARED_SCALE, 1)
    _, gt = gw.build(ctx, w)
    eo, ev = wl.orbital_energies(w)
    deo = torch.tensor(eo, dtype=torch.float64, device="cuda:0")
    dev = torch.tensor(ev, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    ctx.triples_energy(gt["T"], gt["t1"], gt["V_ooov"], gt["V_vovv"], gt["V_oovv"], deo.data_ptr(), dev.data_ptr(),
                       out.data_ptr(), "ozaki_bf16", 6)
    ctx.sync()
    _, ot = O.build_workload(w)
    ref = O.triples_energy(ot, eo, ev)
    err = abs(float(out.item()) - ref) / abs(ref)
    print(f"(T) shared scaling: {err:.2e}")
    assert err <= 1e-10
