"""Pins for the oracle's perturbative triples correction (Sec. IV.B, Eqs. cc14, tensort, tensort2).

None of them retypes the eighteen-term list of Eq. tensort.  W is rebuilt from one base product per
group as its full antisymmetriser over the occupied and the virtual triple,

    A = 1/4 Asym[ sum_m v^{ij}_{ma} t^{mk}_{bc} ],   B = -1/4 Asym[ sum_e v^{ei}_{ab} t^{jk}_{ec} ],
    Y = 1/4 Asym[ v^{ij}_{ab} t^k_c ],               Asym F = sum_{s, t in S3} sgn(s) sgn(t) F(s(ijk), t(abc)),

(each base product is antisymmetric in one occupied and one virtual pair, so the 36 signed
permutations repeat each of the nine distinct terms four times): W must be antisymmetric in the
occupied and the virtual triple, which fixes every sign of Eq. tensort.  Then

* the oracle's W and Y of single triples equal the antisymmetrised construction;
* its restricted sum over i<j<k, a<b<c equals the unrestricted sum over all index tuples / 36;
* W vanishes where spin is not conserved;
* E is quadratic in T2 at t1 = 0, its t1 part linear, and odd in the orbital energies;
* planted mistakes (the sixth term's sign as printed, a dropped term, a wrong restriction, a
  wrong Y sign) fail these pins.
"""
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from tamm_synth import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def _sign(p):
    s, p = 1, list(p)
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def _asym(F):
    """Sum over the 36 signed permutations of the occupied axes (0,1,2) and virtual axes (3,4,5)."""
    out = np.zeros_like(F)
    for so in itertools.permutations(range(3)):
        for sv in itertools.permutations(range(3)):
            out += _sign(so) * _sign(sv) * np.transpose(F, list(so) + [3 + x for x in sv])
    return out


def _tiny(seed_k=7, O_=6, V_=8):
    w = wl.triples(O_, V_, 1, 2, seed_k)
    _, T = O.build_workload(w)
    eo, ev = wl.orbital_energies(w)
    return w, T, eo, ev


def _dense_wy(T):
    vo, vv, voo = T["V_ooov"].to_dense(), T["V_vovv"].to_dense(), T["V_oovv"].to_dense()
    t2, t1 = T["T"].to_dense(), T["t1"].to_dense()
    X = np.einsum("ijma,bcmk->ijkabc", vo, t2)
    Z = np.einsum("eiab,ecjk->ijkabc", vv, t2)
    y0 = np.einsum("ijab,ck->ijkabc", voo, t1)
    return 0.25 * _asym(X) - 0.25 * _asym(Z), 0.25 * _asym(y0)


def _denominators(eo, ev):
    return (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None] +
            eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None] -
            ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])


def _pins_hold() -> bool:
    try:
        w, T, eo, ev = _tiny()
        W, Y = _dense_wy(T)
        # W and Y of single triples, ordered and not
        for (i, j, k) in ((0, 1, 2), (1, 3, 5), (4, 0, 2)):
            wo, yo = O.triples_wy(T, i, j, k)
            scale = np.abs(W).max()
            if np.abs(wo - W[i, j, k]).max() > 1e-14 * scale or np.abs(yo - Y[i, j, k]).max() > 1e-14 * np.abs(Y).max():
                return False
        E = O.triples_energy(T, eo, ev)
        E_all = float(np.sum((W + Y) * W / _denominators(eo, ev))) / 36.0
        return abs(E - E_all) <= 1e-12 * abs(E_all) and E_all != 0.0
    except O.OracleError:
        return False


def test_antisymmetrised_construction_is_antisymmetric():
    _, T, _, _ = _tiny()
    W, Y = _dense_wy(T)
    for X in (W, Y):
        tol = 1e-14 * np.abs(X).max()  # the permuted sums round in different orders
        assert tol > 0
        np.testing.assert_allclose(X, -np.transpose(X, (1, 0, 2, 3, 4, 5)), rtol=0, atol=tol)
        np.testing.assert_allclose(X, -np.transpose(X, (0, 2, 1, 3, 4, 5)), rtol=0, atol=tol)
        np.testing.assert_allclose(X, -np.transpose(X, (0, 1, 2, 4, 3, 5)), rtol=0, atol=tol)
        np.testing.assert_allclose(X, -np.transpose(X, (0, 1, 2, 3, 5, 4)), rtol=0, atol=tol)


def test_oracle_matches_antisymmetrised_construction():
    assert _pins_hold()


def test_spin_conservation_zeros():
    w, T, _, _ = _tiny()
    so = np.array([t[2] for t in T["T"].modes[2].tiles for _ in range(t[1])])
    sv = np.array([t[2] for t in T["T"].modes[0].tiles for _ in range(t[1])])
    nz = 0
    for (i, j, k) in ((0, 1, 2), (0, 1, 4), (0, 4, 5), (3, 4, 5)):
        wo, yo = O.triples_wy(T, i, j, k)
        allowed = (sv[:, None, None] + sv[None, :, None] + sv[None, None, :]) == so[i] + so[j] + so[k]
        assert not wo[~allowed].any() and not yo[~allowed].any()
        nz += int(np.count_nonzero(wo[allowed]))
    assert nz > 0


def test_scaling_invariants():
    w, T, eo, ev = _tiny(seed_k=8)
    t2, t1 = T["T"].data.copy(), T["t1"].data.copy()

    def E(lam, mu, sign=1.0):
        T["T"].data[:] = lam * t2
        T["t1"].data[:] = mu * t1
        return O.triples_energy(T, sign * eo, sign * ev)

    e10, e20, e11, e21 = E(1, 0), E(2, 0), E(1, 1), E(2, 1)
    assert e10 < 0  # every denominator is negative and the W W part is a sum of squares over D
    assert abs(e20 - 4 * e10) <= 1e-13 * abs(e20)
    assert abs((e21 - e20) - 2 * (e11 - e10)) <= 1e-12 * abs(e21 - e20)
    assert abs(E(1, 1, -1.0) + e11) <= 1e-14 * abs(e11)


MUTANTS = {
    "sixth_term_sign_as_printed": ("    s -= VO_(i, k, m, c) * T2_(a, b, m, j);", "    s += VO_(i, k, m, c) * T2_(a, b, m, j);"),
    "drop_b_term": ("    s += VV_(e, j, b, c) * T2_(e, a, i, k);\n", ""),
    "restriction_b_unrestricted": ("for (int64_t b = a + 1; b < nv; ++b)\n        for (int64_t c = b + 1",
                                   "for (int64_t b = 0; b < nv; ++b)\n        for (int64_t c = b + 1"),
    "y_sign": ("VOO_(i, k, a, c) * T1_(b, j) - VOO_(i, k, b, c)", "VOO_(i, k, a, c) * T1_(b, j) + VOO_(i, k, b, c)"),
    "w_counted_once_only": ("s += (w + y) * w / d;", "s += y * w / d;"),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_triples_mistakes(mutant, tmp_path):
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "tamm_oracle.c")).read()
    old, new = MUTANTS[mutant]
    assert src.count(old) == 1, mutant
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", str(path), "-o", str(lib), "-lm"])
    assert _pins_hold()
    with O.using_library(str(lib)):
        caught = not _pins_hold()
    assert caught, f"planted mistake {mutant!r} was not caught"
