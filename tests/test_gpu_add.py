"""Permuted adds (AddOp with label permutation, Sec. III.A grammar rule alpha * A) on both kernel paths:
the chunked path (every term reads the destination's last mode contiguously) and the tiled path (terms
that read it with a stride are staged through shared memory in 32 x 32 tiles of a transposed plane).

Against the oracle's add, one term at a time, on even and ragged tiles, 1 to 4 terms, beta 0 and 1,
alpha +-1 (copies move bits only) and general: relative error <= 1e-15 (a sum of terms rounds once per
term on both sides, in a different order for several terms); a single term with alpha = +-1 is exact.
"""
import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

from parity import gpu_to_oracle_layout, oracle_to_gpu_layout, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # (lc, [(alpha, la), ...], beta)
    ("abij", [(1.0, "abij")], 0.0),                                     # copy: chunked, exact
    ("abij", [(-1.0, "abji")], 0.0),                                    # transposed copy: tiled, exact
    ("abij", [(1.0, "baji")], 1.0),                                     # tiled, accumulate
    ("abij", [(0.7, "abij"), (-1.3, "baij")], 1.0),                     # two chunked terms
    ("abij", [(1.0, "abij"), (-1.0, "baij"), (-1.0, "abji"), (1.0, "baji")], 1.0),  # P(ab)P(ij)
    ("abij", [(2.5, "ijab")], 0.0),                                     # block transposition (oovv -> vvoo)
]


@pytest.fixture(scope="module", params=[(8, 24, 2, 4), (10, 34, 4, 7), (40, 80, 20, 40)],
                ids=["even", "ragged", "wide"])
def spaces(request):
    import paper_2201_01257_gb300 as tg

    O_, V_, to, tv = request.param
    w = wl.small_doubles(O_, V_, to, tv)
    ctx = tg.Context(0)
    gs = {k: ctx.space(s.groups, s.tile, s.tile_sizes) for k, s in w.spaces.items()}
    os_ = {k: O.Space.from_spec(s) for k, s in w.spaces.items()}
    return ctx, gs, os_


@pytest.mark.parametrize("case", range(len(CASES)))
def test_permuted_add_matches_oracle(spaces, case):
    ctx, gs, os_ = spaces
    lc, terms, beta = CASES[case]
    rng = np.random.default_rng(case)
    v, o = "virt", "occ"
    src_modes = {"abij": (v, v, o, o), "ijab": (o, o, v, v)}
    la0 = terms[0][1]
    smodes = src_modes["ijab" if la0 == "ijab" else "abij"]
    A_o = O.Tensor([os_[m] for m in smodes], 2)
    A_o.data[:] = rng.standard_normal(A_o.n_elems)
    C_o = O.Tensor([os_[m] for m in (v, v, o, o)], 2)
    C_o.data[:] = rng.standard_normal(C_o.n_elems)
    A = ctx.tensor([gs[m] for m in smodes], 2)
    C = ctx.tensor([gs[m] for m in (v, v, o, o)], 2)
    A.upload(oracle_to_gpu_layout(A_o, A_o.data, A))
    C.upload(oracle_to_gpu_layout(C_o, C_o.data, C))
    ctx.add(C, lc, beta, A, terms)
    ctx.sync()
    got = gpu_to_oracle_layout(C, C_o)
    for t, (alpha, la) in enumerate(terms):
        O.add(alpha, C_o, lc, beta if t == 0 else 1.0, A_o, la)
    err = rel_err(got, C_o.data)
    print(case, f"{err:.2e}")
    if len(terms) == 1 and abs(terms[0][0]) == 1.0:
        assert np.array_equal(got, C_o.data), case
    assert err <= 1e-15, (case, err)
