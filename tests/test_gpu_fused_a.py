"""The split-precision GEMM that slices its A operand itself (block pairs summing at most 48 indices, output
blocks of at most 64 columns), on the singles term of the CCSD doubles residual,
R[a,b,i,j] = beta R + alpha sum_e V[a,b,e,j] t1[e,i], against the FP64 oracle and against the pre-sliced
path (TAMM_OPT_OZAKI_FUSED_A = 0).

Shapes cover ragged row tiles (M not a multiple of 128), K not a multiple of 16 and exactly 48, output
widths N from 2 to 64 (one to four accumulator buffers), the output permutation abji -> abij written through
C's strides, and alpha/beta combinations (alpha a power of two folded into the exponent, or not; beta 0 or
1).  A contraction with 56 summed indices per block pair stays on the pre-sliced path."""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def t1_workload(O_, V_, to, tv, alpha, beta):
    w = wl._vt(11, O_, V_, to, tv, f"t1_O{O_}_V{V_}")
    w.tensors = {
        "V_vvvo": wl.TensorSpec("V_vvvo", ("virt", "virt", "virt", "occ"), 2, sigma=0.1, stream=6, anti01=True),
        "t1": wl.TensorSpec("t1", ("virt", "occ"), 1, sigma=0.01, stream=7),
        "T": wl.TensorSpec("T", ("virt", "virt", "occ", "occ"), 2, sigma=0.01, stream=2, anti01=True, anti23=True),
        "R": wl.TensorSpec("R", ("virt", "virt", "occ", "occ"), 2),
    }
    w.steps = [
        wl.AddSpec("seed", "R", "abij", "T", "abij", 1.0, beta=0.0),
        wl.ContractSpec("t1", "R", "abij", "V_vvvo", "abej", "t1", "ei", alpha, beta=beta),
    ]
    return w


def run_gpu(tg, w, fused):
    from paper_2201_01257_gb300 import workload as gw

    ctx = tg.Context(0)
    ctx.set_option(tg.TAMM_OPT_OZAKI_FUSED_A, 1 if fused else 0)
    gsp, gt = gw.build(ctx, w)
    run = gw.Runner(ctx, w, gsp, gt)
    run.run("f64", 0, steps=[w.steps[0]])
    ctx.sync()
    ctx.profile_read()
    ctx.profile(True)
    run.run("ozaki_bf16", 6, steps=[w.steps[1]])
    ctx.sync()
    ctx.profile(False)
    prof = ctx.profile_read()
    return gt, prof


# (O, V, occupied tile, virtual tile): N = occupied tile, K = virtual tile, M = tv^2 * to rows per block
CASES = [
    (8, 24, 2, 4),
    (10, 34, 4, 7),
    (20, 80, 10, 40),
    (24, 96, 12, 48),
    (96, 64, 48, 32),
    (128, 48, 64, 24),
]
SCALES = [(1.0, 1.0), (0.3, 1.0), (-2.0, 0.0)]


@pytest.mark.parametrize("shape", CASES, ids=lambda s: "O%d_V%d_t%d_%d" % s)
@pytest.mark.parametrize("alpha,beta", SCALES, ids=["a1_b1", "a0.3_b1", "a-2_b0"])
def test_fused_a_singles_term(gpu_lib, shape, alpha, beta):
    w = t1_workload(*shape, alpha, beta)
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    ref = ot["R"].data
    out = {}
    for fused in (True, False):
        gt, prof = run_gpu(gpu_lib, w, fused)
        got = gpu_to_oracle_layout(gt["R"], ot["R"])
        err = rel_err(got, ref)
        assert err <= TOL, (fused, err)
        # the fused path slices only B (one slicing launch); the pre-sliced path slices A and B
        assert prof["slice"][1] == (1 if fused else 2), (fused, prof["slice"])
        out[fused] = got
    # both paths carry the same digits; only the order of the exact-chunk folds' references differs
    assert rel_err(out[True], out[False]) <= 1e-13


def test_long_k_stays_presliced(gpu_lib):
    """56 summed indices per block pair (> 48): the pre-sliced path runs, A and B sliced separately."""
    w = t1_workload(8, 112, 4, 56, 1.0, 1.0)
    _, ot = O.build_workload(w)
    O.run_workload(w, ot)
    gt, prof = run_gpu(gpu_lib, w, True)
    assert rel_err(gpu_to_oracle_layout(gt["R"], ot["R"]), ot["R"].data) <= TOL
    assert prof["slice"][1] == 2, prof["slice"]
