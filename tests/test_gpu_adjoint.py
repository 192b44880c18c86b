"""tamm_contract_adjoint through the C ABI: the adjoint of a MultOp (Sec. III.A, grammar figure
"tensor_ops") is a MultOp with the label roles exchanged,

    dA(la) = beta dA + alpha sum dC(lc) B(lb),   dB(lb) = beta dB + alpha sum A(la) dC(lc),

checked against the oracle running those exchanged-role contractions on the same seeded inputs
(FP64 <= 1e-12, split precision <= 1e-10), for the ladder (no operand permutation) and the ring
term (both operands permuted), plus the refusals of the call.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, oracle_to_gpu_layout, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "ladder": ("R", "abij", "V_vvvv", "abef", "T", "efij", 0.5),
    "ring": ("R", "abij", "T", "aeim", "V_ovvo", "mbej", 1.0),
    "t1": ("R", "abij", "V_vvvo", "abej", "t1", "ei", 1.0),
}


@pytest.fixture(scope="module")
def small():
    import paper_2201_01257_gb300 as tg
    from paper_2201_01257_gb300 import workload as gw

    w = wl.small_doubles(O=8, V=24, to=2, tv=4)
    ctx = tg.Context(0)
    _, gt = gw.build(ctx, w)
    _, ot = O.build_workload(w)
    return ctx, gt, ot


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("ozaki_bf16", 1e-10)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_matches_oracle_exchanged_roles(small, case, precision, tol):
    ctx, gt, ot = small
    c, lc, a, la, b, lb, alpha = CASES[case]
    rng = np.random.default_rng(11)
    # incoming adjoint dC with C's block structure, random entries
    dC_o = O.Tensor(ot[c].modes, ot[c].n_upper)
    dC_o.data[:] = rng.standard_normal(dC_o.n_elems)
    dC = ctx.tensor_permuted(gt[c], list(range(gt[c].nm)))
    dC.upload(oracle_to_gpu_layout(dC_o, dC_o.data, dC))
    # dA and dB start from seeded values and accumulate (beta = 1)
    dA_o = O.Tensor(ot[a].modes, ot[a].n_upper)
    dB_o = O.Tensor(ot[b].modes, ot[b].n_upper)
    dA_o.data[:] = rng.standard_normal(dA_o.n_elems)
    dB_o.data[:] = rng.standard_normal(dB_o.n_elems)
    dA = ctx.tensor_permuted(gt[a], list(range(gt[a].nm)))
    dB = ctx.tensor_permuted(gt[b], list(range(gt[b].nm)))
    dA.upload(oracle_to_gpu_layout(dA_o, dA_o.data, dA))
    dB.upload(oracle_to_gpu_layout(dB_o, dB_o.data, dB))
    ctx.contract_adjoint(alpha, dC, lc, gt[a], la, gt[b], lb, dA=dA, dB=dB, beta=1.0, precision=precision)
    ctx.sync()
    O.contract(alpha, dA_o, la, 1.0, dC_o, lc, ot[b], lb)
    O.contract(alpha, dB_o, lb, 1.0, ot[a], la, dC_o, lc)
    for name, G, R in (("dA", dA, dA_o), ("dB", dB, dB_o)):
        err = rel_err(gpu_to_oracle_layout(G, R), R.data)
        print(f"{case} {precision} {name}: {err:.2e}")
        assert err <= tol, (case, precision, name, err)


def test_adjoint_one_side_and_overwrite(small):
    # dB = NULL computes dA alone; beta = 0 overwrites whatever dA held
    import torch

    ctx, gt, ot = small
    dA = ctx.tensor_permuted(gt["V_vvvv"], [0, 1, 2, 3])
    dA.data.fill_(float("nan"))
    ctx.contract_adjoint(0.5, gt["R"], "abij", gt["V_vvvv"], "abef", gt["T"], "efij", dA=dA, beta=0.0)
    ref = ctx.tensor_permuted(gt["V_vvvv"], [0, 1, 2, 3])
    ctx.contract(0.5, ref, "abef", 0.0, gt["R"], "abij", gt["T"], "efij")
    ctx.sync()
    assert torch.equal(dA.data, ref.data)


def test_adjoint_refusals(small):
    import paper_2201_01257_gb300 as tg

    ctx, gt, _ = small
    dT = ctx.tensor_permuted(gt["T"], [0, 1, 2, 3])
    other = ctx.tensor_permuted(gt["V_oovv"], [0, 1, 2, 3])  # other spaces: another block table
    for kwargs in ({}, {"dB": other}, {"dA": dT}):
        with pytest.raises(tg.TammError) as e:
            ctx.contract_adjoint(0.5, gt["R"], "abij", gt["V_vvvv"], "abef", gt["T"], "efij", **kwargs)
        assert e.value.status == tg.TAMM_EINVAL
    with pytest.raises(tg.TammError) as e:  # the forward's labels are invalid (k only in B)
        ctx.contract_adjoint(0.5, gt["R"], "abij", gt["V_vvvv"], "abef", gt["T"], "efkj", dB=dT)
    assert e.value.status == tg.TAMM_EINVAL
    with pytest.raises(tg.TammError) as e:
        ctx.contract_adjoint(0.5, gt["R"], "abij", gt["V_vvvv"], "abef", gt["T"], "efij", dB=dT, beta=0.5)
    assert e.value.status == tg.TAMM_EINVAL
