"""Autotuner of the split-precision path (slice count and exact-chunk length).

On the O=32 V=192 ladder (tiles 16/32) and a small doubles ring (output permutation):
* the chosen configuration meets the target against the FP64 oracle itself (not only against the
  GPU's FP64 reference the tuner used), on seeded sub-blocks;
* a looser target never needs more slices than a tighter one;
* tamm_contract with slices = 0 then runs the tuned configuration: bitwise equal to the same slice
  count and chunk length given explicitly;
* C's own data is not touched by tuning; an unreachable target is refused with TAMM_EUNSUPPORTED.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ladder_energy():
    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.ladder_energy_o32_v192()
    ctx = tg.Context(0)
    gsp, gt = gw.build(ctx, w, only={"V_vvvv", "T", "Tp"})
    return tg, ctx, w, gt


def sampled_error(R_gpu, ot, n=64, seed=11):
    """Normwise error of Tp = 0.5 V_vvvv T over seeded 4^4 sub-blocks computed by the oracle."""
    R = ot["Tp"]
    rng = np.random.default_rng(seed)
    _, ext = R.block_lo_ext()
    bl = rng.integers(R.n_blocks, size=n)
    lo = [[int(rng.integers(0, e - 3)) for e in ext[b]] for b in bl]
    vals = O.contract_boxes(0.5, R, "abij", ot["V_vvvv"], "abef", ot["T"], "efij", bl, lo, [[4] * 4] * n)
    got = gpu_to_oracle_layout(R_gpu, R)
    num = den = 0.0
    for b, l, v in zip(bl, lo, vals):
        blk = got[R.block_off[b]:R.block_off[b] + int(np.prod(ext[b]))].reshape(tuple(ext[b]))
        sub = blk[l[0]:l[0] + 4, l[1]:l[1] + 4, l[2]:l[2] + 4, l[3]:l[3] + 4]
        num += float(np.sum((sub - v) ** 2))
        den += float(np.sum(v ** 2))
    return float(np.sqrt(num / den))


def test_autotune_meets_target_and_is_used(ladder_energy):
    tg, ctx, w, gt = ladder_energy
    V, T, R = gt["V_vvvv"], gt["T"], gt["Tp"]
    R.data.fill_(7.0)
    ctx.sync()
    tight = ctx.autotune(R, "abij", V, "abef", T, "efij", 1e-10)
    loose = ctx.autotune(R, "abij", V, "abef", T, "efij", 1e-4)
    ctx.sync()
    assert np.all(R.download() == 7.0)  # tuning leaves C alone
    print("autotune 1e-10:", tight, " 1e-4:", loose)
    assert tight["rel_err"] <= 0.5e-10 and loose["rel_err"] <= 0.5e-4
    assert loose["slices"] <= tight["slices"]
    assert 3 <= tight["slices"] <= 8 and tight["chunk_k"] in (320, 640, 800, 1280)
    assert tight["tile_policy"] in (0, 1, 2, 3)
    # the last tuning (1e-4) is the remembered one: re-tune at 1e-10 and use it through slices = 0
    tight = ctx.autotune(R, "abij", V, "abef", T, "efij", 1e-10)
    ctx.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij", "ozaki_bf16", 0)
    auto = R.download()
    ctx.set_option(tg.TAMM_OPT_OZAKI_CHUNK_K, tight["chunk_k"])
    ctx.set_option(tg.TAMM_OPT_OZAKI_TILE_POLICY, tight["tile_policy"])
    ctx.set_option(tg.TAMM_OPT_OZAKI_PERSISTENT, tight["persistent"])
    ctx.set_option(tg.TAMM_OPT_OZAKI_SHARED_SCALE, tight["shared_scale"])
    ctx.set_option(tg.TAMM_OPT_OZAKI_FUSED_A, tight["fused_a"])
    ctx.contract(0.5, R, "abij", 0.0, V, "abef", T, "efij", "ozaki_bf16", tight["slices"])
    explicit = R.download()
    ctx.set_option(tg.TAMM_OPT_OZAKI_CHUNK_K, 640)
    ctx.set_option(tg.TAMM_OPT_OZAKI_TILE_POLICY, 1)
    ctx.set_option(tg.TAMM_OPT_OZAKI_PERSISTENT, 0)
    ctx.set_option(tg.TAMM_OPT_OZAKI_SHARED_SCALE, 0)
    ctx.set_option(tg.TAMM_OPT_OZAKI_FUSED_A, 0)
    assert np.array_equal(auto, explicit)
    _, ot = O.build_workload(wl.Workload(w.name, w.seed, w.spaces,
                                         {k: w.tensors[k] for k in ("V_vvvv", "T", "Tp")}))
    err = sampled_error(R, ot)
    print(f"tuned ladder vs oracle: {err:.3e}")
    assert err <= 1e-10


def test_autotune_ring_with_output_permutation(gpu_lib):
    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles(16, 40, 8, 10)
    ctx = gpu_lib.Context(0)
    gsp, gt = gw.build(ctx, w)
    runner = gw.Runner(ctx, w, gsp, gt)
    ring = next(s for s in w.steps if s.name == "ring")
    X, lx = runner.scratch_for(ring)
    r = ctx.autotune(X, lx, gt[ring.a], ring.la, gt[ring.b], ring.lb, 1e-10)
    assert r["rel_err"] <= 0.5e-10
    runner.run("ozaki_bf16", 0)
    ctx.sync()
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    for name in ("R", "W"):
        assert rel_err(gpu_to_oracle_layout(gt[name], ot[name]), ot[name].data) <= 1e-10, name


def test_autotune_unreachable_target(ladder_energy):
    tg, ctx, w, gt = ladder_energy
    with pytest.raises(tg.TammError) as e:
        ctx.autotune(gt["Tp"], "abij", gt["V_vvvv"], "abef", gt["T"], "efij", 1e-30)
    assert e.value.status == tg.TAMM_EUNSUPPORTED
    with pytest.raises(tg.TammError) as e:
        ctx.autotune(gt["Tp"], "abij", gt["V_vvvv"], "abef", gt["T"], "efij", -1.0)
    assert e.value.status == tg.TAMM_EINVAL


def test_autotune_refuses_a_zero_product(ladder_energy):
    import torch

    tg, ctx, w, gt = ladder_energy
    zero = torch.zeros_like(gt["T"].data)
    Tz = ctx.tensor_permuted(gt["T"], [0, 1, 2, 3], allocate=False)
    Tz.bind(zero)
    with pytest.raises(tg.TammError) as e:
        ctx.autotune(gt["Tp"], "abij", gt["V_vvvv"], "abef", Tz, "efij", 1e-10)
    assert e.value.status == tg.TAMM_EINVAL and "zero" in str(e.value)
