"""Pins for the oracle's Cholesky-built two-electron tensor (Eq. cc12).

V[p,q,r,s] = sum_L X[p,r,L] X[q,s,L] - X[p,s,L] X[q,r,L], X with modes (P, R, aux) and a spinless
auxiliary index.  Pinned against dense ``numpy.einsum`` on tiny inputs (ragged tiles, several aux
tiles, equal and different P/R spaces), closed forms (identity vectors give the antisymmetrised
identity, one rank-one vector gives zero), the exact symmetries the formula implies, and storage
counts.  The mutation tests compile broken copies of the oracle and check that a pin catches each.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
import tamm_synth
from tamm_synth import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def spin_space(n, tile):
    return O.Space([(n // 2, 1, 0), (n // 2, -1, 0)], tile)


def aux(n, tile):
    return O.Space([(n, 0, 0)], tile)


def random_x(P, R, L, seed, symmetric=False):
    X = O.Tensor([P, R, L], 1)
    d = np.random.default_rng(seed).standard_normal(X.dense_shape())
    if symmetric:
        d = d + d.transpose(1, 0, 2)
    X.from_dense(d)
    return X


def formed(X):
    P, R = X.modes[0], X.modes[1]
    V = O.Tensor([P, P, R, R], 2)
    O.cholesky_v(V, X)
    return V


def einsum_v(Xd):
    return np.einsum("prL,qsL->pqrs", Xd, Xd) - np.einsum("psL,qrL->pqrs", Xd, Xd)


@pytest.mark.parametrize("p_n,p_tile,r_n,r_tile,n_aux,aux_tile", [
    (12, 4, 12, 4, 7, 3),    # virt-virt, ragged spin groups (6 = 4 + 2), aux tiles 3, 3, 1
    (6, 2, 10, 3, 5, 5),     # occ-virt (V_oovv-shaped), one aux tile
    (8, 3, 8, 3, 9, 2),      # tiles 3, 1 per group, five aux tiles
])
def test_cholesky_v_matches_dense_einsum(p_n, p_tile, r_n, r_tile, n_aux, aux_tile):
    P, R, L = spin_space(p_n, p_tile), spin_space(r_n, r_tile), aux(n_aux, aux_tile)
    X = random_x(P, R, L, seed=p_n * 100 + n_aux)
    Xd = X.to_dense()
    # spinless aux index: X stores exactly the spin-diagonal (p, r) pairs
    assert X.n_elems == 2 * (p_n // 2) * (r_n // 2) * n_aux
    V = formed(X)
    ref = einsum_v(Xd)
    # every entry outside the stored blocks of V is zero in the dense result, every stored entry matches
    assert np.allclose(V.to_dense(), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.abs(ref).max() > 1.0


def test_cholesky_v_exact_symmetries():
    v = spin_space(12, 4)
    X = random_x(v, v, aux(10, 4), seed=3, symmetric=True)
    Vd = formed(X).to_dense()
    assert np.array_equal(Vd, -Vd.transpose(1, 0, 2, 3))  # p <-> q
    assert np.array_equal(Vd, -Vd.transpose(0, 1, 3, 2))  # r <-> s
    assert np.array_equal(Vd, Vd.transpose(2, 3, 0, 1))   # (pq) <-> (rs) when X[p,r] = X[r,p]
    assert np.all(Vd[np.arange(12), np.arange(12)] == 0.0)


def test_cholesky_v_identity_vectors_give_antisymmetrised_identity():
    # one vector X[p,r,0] = delta_pr: V[p,q,r,s] = delta_pr delta_qs - delta_ps delta_qr
    v = spin_space(8, 2)
    X = O.Tensor([v, v, aux(1, 1)], 1)
    X.from_dense(np.eye(8)[:, :, None])
    e = np.eye(8)
    closed = np.einsum("pr,qs->pqrs", e, e) - np.einsum("ps,qr->pqrs", e, e)
    assert np.array_equal(formed(X).to_dense(), closed)


def test_cholesky_v_rank_one_vector_closed_form():
    # one vector X[p,r,0] = u_p u_r S_pr (S = 1 for equal spins, the spinless aux index keeps only those):
    # V[p,q,r,s] = u_p u_q u_r u_s (S_pr S_qs - S_ps S_qr), zero when all four spins are equal
    v = spin_space(8, 4)
    u = np.random.default_rng(5).standard_normal(8)
    spin = np.array([1] * 4 + [-1] * 4)
    S = (spin[:, None] == spin[None, :]).astype(float)
    X = O.Tensor([v, v, aux(1, 1)], 1)
    X.from_dense((np.outer(u, u) * S)[:, :, None])
    Vd = formed(X).to_dense()
    u4 = np.einsum("p,q,r,s->pqrs", u, u, u, u)
    closed = u4 * (np.einsum("pr,qs->pqrs", S, S) - np.einsum("ps,qr->pqrs", S, S))
    scale = np.abs(u).max() ** 4
    assert np.allclose(Vd, closed, rtol=0, atol=1e-15 * scale)
    assert np.abs(Vd[:4, :4, :4, :4]).max() <= 1e-15 * scale
    assert np.abs(closed).max() > 0.1 * scale


def test_cholesky_v_listed_blocks_only():
    v = spin_space(12, 4)
    X = random_x(v, v, aux(7, 3), seed=8)
    full = formed(X)
    part = O.Tensor([v, v, v, v], 2)
    part.data[:] = 5.0
    listed = [0, 7, full.n_blocks - 1]
    O.cholesky_v(part, X, listed)
    for b in range(full.n_blocks):
        got, want = part.block_view(b), full.block_view(b)
        if b in listed:
            assert np.array_equal(got, want)
        else:
            assert np.all(got == 5.0)


def test_cholesky_v_rejects_mismatched_spaces():
    v, o = spin_space(8, 4), spin_space(4, 2)
    X = random_x(v, v, aux(4, 2), seed=1)
    bad = O.Tensor([v, o, v, v], 2)
    with pytest.raises(O.OracleError):
        O.cholesky_v(bad, X)


def test_synthetic_cholesky_vectors_are_symmetric():
    w = wl.cholesky_ladder_o8_v32()
    _, t = O.build_workload(w)
    Xd = t["X"].to_dense()
    assert np.array_equal(Xd, Xd.transpose(1, 0, 2))
    # alpha-beta pairs are not stored (spinless aux index); stored off-diagonal entries have std sigma
    half = 16
    assert np.all(Xd[:half, half:] == 0.0) and np.all(Xd[half:, :half] == 0.0)
    sigma = w.tensors["X"].sigma
    off = Xd[:half, :half][~np.eye(half, dtype=bool)]
    assert abs(np.std(off) / sigma - 1.0) < 0.05
    # each stored entry is the symmetrised pair of the generator's plain draws
    plain = np.zeros(1)
    tamm_synth.fill_boxes(w.seed, 8, sigma, Xd.shape, False, False, [[3, 5, 7]], [[1, 1, 1]], [0], plain)
    other = np.zeros(1)
    tamm_synth.fill_boxes(w.seed, 8, sigma, Xd.shape, False, False, [[5, 3, 7]], [[1, 1, 1]], [0], other)
    assert Xd[3, 5, 7] == (plain[0] + other[0]) * 0.70710678118654752440 or \
        abs(Xd[3, 5, 7] - (plain[0] + other[0]) / np.sqrt(2.0)) <= 1e-16


def test_cholesky_ladder_recipe_matches_dense():
    w = wl.cholesky_ladder_o8_v32()
    _, t = O.build_workload(w)
    O.run_workload(w, t)
    Vd = einsum_v(t["X"].to_dense())
    ref = 0.5 * np.einsum("abef,efij->abij", Vd, t["T"].to_dense())
    got = t["R"].to_dense()
    assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.abs(ref).max() > 1e-3


# --------------------------------------------------------- mutation tests

MUTANTS = {
    "second_term_sign": ("acc += x_pr * x_qs - x_ps * x_qr;", "acc += x_pr * x_qs + x_ps * x_qr;"),
    "second_term_dropped": ("acc += x_pr * x_qs - x_ps * x_qr;", "acc += x_pr * x_qs;"),
    "swapped_index": ("x[X->off[b_ps] + (ip * ns + is) * nl + l]", "x[X->off[b_ps] + (is * np + ip) * nl + l]"),
    "last_vector_dropped": ("for (int64_t l = 0; l < nl; ++l) {", "for (int64_t l = 0; l + 1 < nl; ++l) {"),
    "first_aux_tile_only": ("for (int tl = 0; tl < aux->n_tiles; ++tl) {", "for (int tl = 0; tl < 1; ++tl) {"),
    "wrong_partner": ("acc += x_pr * x_qs - x_ps * x_qr;", "acc += x_pr * x_qr - x_ps * x_qs;"),
}


def _pins_hold() -> bool:
    try:
        P, R, L = spin_space(6, 2), spin_space(10, 3), aux(5, 2)
        X = random_x(P, R, L, seed=11)
        ref = einsum_v(X.to_dense())
        if not np.allclose(formed(X).to_dense(), ref, rtol=0, atol=1e-13 * np.abs(ref).max()):
            return False
        v = spin_space(12, 4)
        Vd = formed(random_x(v, v, aux(10, 4), seed=3, symmetric=True)).to_dense()
        return bool(np.array_equal(Vd, -Vd.transpose(1, 0, 2, 3)) and np.array_equal(Vd, Vd.transpose(2, 3, 0, 1)))
    except (O.OracleError, IndexError):
        return False


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_cholesky_mistakes(mutant, tmp_path):
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "tamm_oracle.c")).read()
    old, new = MUTANTS[mutant]
    assert src.count(old) == 1, mutant
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", str(path), "-o", str(lib), "-lm"])
    assert _pins_hold()
    with O.using_library(str(lib)):
        caught = not _pins_hold()
    assert caught, f"planted mistake {mutant!r} was not caught"


def test_oracle_cholesky_regression_values():
    import json

    g = json.load(open(os.path.join(HERE, "golden", "oracle_cholesky_ladder_o8_v32.json")))
    w = wl.cholesky_ladder_o8_v32()
    _, t = O.build_workload(w)
    O.run_workload(w, t)
    assert t["X"].n_elems == g["n_elems_X"] and t["V_chol"].n_elems == g["n_elems_V"]
    for key, val in (("norm_X", O.norm(t["X"])), ("norm_V", O.norm(t["V_chol"])), ("norm_R", O.norm(t["R"])),
                     ("R_dot_T", O.energy(1.0, t["R"], "abij", t["T"], "abij"))):
        assert abs(val - g[key]) <= 1e-13 * abs(g[key]), key
