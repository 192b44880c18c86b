"""GPU FP64 path vs the FP64 oracle on the same seeded inputs (normwise rel. err <= 1e-12)."""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu
TOL_F64 = 1e-12


def run_both(tg, w, precision="f64", slices=0):
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w)
    runner = gw.Runner(ctx, w, gsp, gt)
    genergy = runner.run(precision, slices)
    ctx.sync()
    _, ot = O.build_workload(w)
    oenergy = O.run_workload(w, ot)
    return ctx, gt, ot, genergy, oenergy


def test_ladder_o8_v32_f64(gpu_lib):
    ctx, gt, ot, _, _ = run_both(gpu_lib, wl.ladder_o8_v32())
    got = gpu_to_oracle_layout(gt["R"], ot["R"])
    assert rel_err(got, ot["R"].data) <= TOL_F64
    assert np.abs(got - ot["R"].data).max() <= 1e-14 * np.abs(ot["R"].data).max()


@pytest.mark.parametrize("O_,V_,to,tv", [(8, 24, 2, 4), (12, 36, 3, 5), (10, 34, 4, 7)])
def test_small_doubles_all_steps_f64(gpu_lib, O_, V_, to, tv):
    # uneven tile sizes give ragged GEMM tiles (M, N, K not multiples of 64/16)
    w = wl.small_doubles(O_, V_, to, tv)
    ctx, gt, ot, ge, oe = run_both(gpu_lib, w)
    for name in ("R", "W"):
        got = gpu_to_oracle_layout(gt[name], ot[name])
        assert rel_err(got, ot[name].data) <= TOL_F64, name
    assert abs(ge["energy"] - oe["energy"]) <= TOL_F64 * abs(oe["energy"])


def test_norm_and_energy_match_oracle(gpu_lib):
    w = wl.small_doubles(8, 24, 2, 4)
    ctx, gt, ot, _, _ = run_both(gpu_lib, w)
    assert abs(ctx.norm(gt["V_vvvv"]) - O.norm(ot["V_vvvv"])) <= 1e-13 * O.norm(ot["V_vvvv"])
    e = ctx.energy(0.25, gt["V_oovv"], "ijab", gt["T"], "abij")
    assert abs(e - O.energy(0.25, ot["V_oovv"], "ijab", ot["T"], "abij")) <= 1e-13 * abs(e)


def test_beta_zero_overwrites_nan_and_alpha_linearity(gpu_lib):
    import torch

    tg = gpu_lib
    w = wl.small_doubles(8, 24, 2, 4)
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    _, t = gw.build(ctx, w)
    R = t["R"]
    R.data.fill_(float("nan"))
    ctx.contract(0.5, R, "abij", 0.0, t["V_vvvv"], "abef", t["T"], "efij")
    r1 = R.download()
    assert np.isfinite(r1).all()
    ctx.contract(0.5, R, "abij", 1.0, t["V_vvvv"], "abef", t["T"], "efij")
    r2 = R.download()
    np.testing.assert_allclose(r2, 2 * r1, rtol=1e-14, atol=1e-300)
    ctx.contract(-1.0, R, "abij", 1.0, t["V_vvvv"], "abef", t["T"], "efij")
    assert np.abs(R.download()).max() <= 1e-15 * np.abs(r1).max()


def test_errors(gpu_lib):
    tg = gpu_lib
    w = wl.small_doubles(8, 24, 2, 4)
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    _, t = gw.build(ctx, w)
    with pytest.raises(tg.TammError) as e:
        ctx.contract(1.0, t["R"], "abij", 0.5, t["V_vvvv"], "abef", t["T"], "efij")
    assert e.value.status == tg.TAMM_EINVAL
    with pytest.raises(tg.TammError) as e:
        ctx.contract(1.0, t["R"], "abij", 0.0, t["V_vvvv"], "abef", t["T"], "efij", precision="ozaki_i8")
    assert e.value.status == tg.TAMM_EUNSUPPORTED
    with pytest.raises(tg.TammError) as e:
        ctx.contract(1.0, t["T"], "abij", 0.0, t["V_vvvv"], "abef", t["T"], "efij")
    assert e.value.status == tg.TAMM_EINVAL


def test_doubles_o40_v240_sampled_blocks_f64(gpu_lib):
    """Full O=40 V=240 doubles sizes on the GPU; oracle recomputes sampled 4x4x4x4 boxes of the output."""
    tg = gpu_lib
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ccsd_doubles_o40_v240()
    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w, only={"V_vvvv", "T", "R"})
    step = w.steps[0]
    ctx.contract(step.alpha, gt["R"], "abij", 0.0, gt["V_vvvv"], "abef", gt["T"], "efij")
    got = gt["R"].download()
    _, ot = O.build_workload(wl.Workload(w.name, w.seed, w.spaces,
                                          {k: w.tensors[k] for k in ("V_vvvv", "T", "R")}))
    R = ot["R"]
    rng = np.random.default_rng(0)
    idx = {tuple(x): k for k, x in enumerate(gt["R"].block_tiles.tolist())}
    lo_all, ext_all = R.block_lo_ext()
    num = den = 0.0
    for b in rng.choice(R.n_blocks, 6, replace=False):
        ext = ext_all[b]
        lo = [int(rng.integers(0, e - 3)) for e in ext]
        ref = O.contract_box(0.5, R, "abij", 0.0, ot["V_vvvv"], "abef", ot["T"], "efij", int(b), lo, [4] * 4)
        k = idx[tuple(R.block_tiles[b].tolist())]
        blk = got[gt["R"].block_offsets[k]:gt["R"].block_offsets[k] + int(np.prod(ext))].reshape(tuple(ext))
        sub = blk[lo[0]:lo[0] + 4, lo[1]:lo[1] + 4, lo[2]:lo[2] + 4, lo[3]:lo[3] + 4]
        num += float(np.sum((sub - ref) ** 2))
        den += float(np.sum(ref ** 2))
    assert np.sqrt(num / den) <= TOL_F64
