"""Run a synthetic workload recipe (``tamm_synth.workloads``) through the GPU library.

Builds the index spaces and block-sparse tensors of a recipe, fills them with
the shared seeded generator on the host (per stored block) and uploads them,
then executes the recipe's steps with ``tamm_contract`` / ``tamm_add`` /
``tamm_energy``.  A contraction with an output antisymmetriser P(ab)P(ij)
writes its product into a scratch tensor laid out in GEMM order and applies
the four signed permutations in one ``tamm_add`` pass.
"""
from __future__ import annotations

import numpy as np

import tamm_synth
from tamm_synth import workloads as wl

from . import CholeskyTensor, Context, Tensor


def build(ctx: Context, w: wl.Workload, fill: bool = True, only=None, slab_bytes: int = 0):
    """Spaces and tensors of a recipe; a tensor formed from Cholesky vectors becomes a lambda tensor over
    them (slab buffers of at most ``slab_bytes``, 0 = the library's default)."""
    spaces = {k: ctx.space(s.groups, s.tile, s.tile_sizes) for k, s in w.spaces.items()}
    tensors = {}
    for name, t in w.tensors.items():
        if (only is not None and name not in only) or t.cholesky:
            continue
        T = ctx.tensor([spaces[m] for m in t.modes], t.n_upper, t.sym)
        if fill and t.sigma != 0.0:
            fill_tensor(T, w.seed, t)
        tensors[name] = T
    for name, t in w.tensors.items():
        if t.cholesky and (only is None or name in only):
            tensors[name] = ctx.tensor_cholesky(tensors[t.cholesky], slab_bytes)
    return spaces, tensors


def fill_tensor(T: Tensor, seed: int, spec: wl.TensorSpec) -> None:
    host = np.zeros(T.n_elems, dtype=np.float64)
    lo, ext = T.block_lo_ext()
    dims = [m.n for m in T.modes]
    tamm_synth.fill_boxes(seed, spec.stream, spec.sigma, dims, spec.anti01, spec.anti23, lo, ext,
                          T.block_offsets, host, sym01=spec.sym01)
    T.upload(host)


def gemm_order(step: wl.ContractSpec) -> str:
    """Output label order of the block GEMMs: C labels of the operand holding C's first label, then the rest."""
    left = step.la if step.lc[0] in step.la else step.lb
    fl = "".join(c for c in step.lc if c in left)
    fr = "".join(c for c in step.lc if c not in left)
    return fl + fr


def antisym_terms(lc: str, lx: str):
    """tamm_add terms for C(lc) += P(ab)P(ij) X, X stored with labels lx (a permutation of lc = 'abij')."""
    a, b, i, j = lc
    swaps = [({}, 1.0), ({a: b, b: a}, -1.0), ({i: j, j: i}, -1.0), ({a: b, b: a, i: j, j: i}, 1.0)]
    return [(s, "".join(m.get(c, c) for c in lx)) for m, s in swaps]


class Runner:
    """Executes a recipe's steps; scratch tensors for antisymmetrised products are cached."""

    def __init__(self, ctx: Context, w: wl.Workload, spaces, tensors):
        self.ctx, self.w, self.spaces, self.tensors = ctx, w, spaces, tensors
        self._scratch = {}

    def scratch_for(self, step: wl.ContractSpec) -> tuple:
        lx = gemm_order(step)
        if step.name not in self._scratch:
            C = self.tensors[step.c]
            perm = [step.lc.index(c) for c in lx]
            self._scratch[step.name] = (self.ctx.tensor_permuted(C, perm), lx)
        return self._scratch[step.name]

    def flops(self, step) -> float:
        """Nonzero-block flops of a contraction step, with forming a lambda operand once counted in."""
        if not isinstance(step, wl.ContractSpec):
            return 0.0
        T = self.tensors
        form = sum(T[n].form_flops for n in (step.a, step.b) if isinstance(T[n], CholeskyTensor))
        if step.antisym:
            X, lx = self.scratch_for(step)
            return form + self.ctx.flops(X, lx, T[step.a], step.la, T[step.b], step.lb)
        return form + self.ctx.flops(T[step.c], step.lc, T[step.a], step.la, T[step.b], step.lb)

    def energy_slot(self, step, energy_out: int) -> int:
        """Device address of an energy step's result: the k-th energy step of the recipe writes the k-th
        double at ``energy_out``."""
        k = [s.name for s in self.w.steps if isinstance(s, wl.EnergySpec)].index(step.name)
        return energy_out + 8 * k

    def run_step(self, step, precision="f64", slices: int = 0, energy_out=None):
        T, ctx = self.tensors, self.ctx
        if isinstance(step, wl.EnergySpec):
            if energy_out is not None:
                ctx.energy_async(step.alpha, T[step.a], step.la, T[step.b], step.lb,
                                 self.energy_slot(step, energy_out))
                return None
            return ctx.energy(step.alpha, T[step.a], step.la, T[step.b], step.lb)
        if isinstance(step, wl.AddSpec):
            ctx.add(T[step.c], step.lc, step.beta, T[step.a], step.terms)
            return None
        if step.antisym:
            X, lx = self.scratch_for(step)
            ctx.contract(step.alpha, X, lx, 0.0, T[step.a], step.la, T[step.b], step.lb, precision, slices)
            ctx.add(T[step.c], step.lc, step.beta, X, antisym_terms(step.lc, lx))
            return None
        ctx.contract(step.alpha, T[step.c], step.lc, step.beta, T[step.a], step.la, T[step.b], step.lb,
                     precision, slices)
        return None

    def run(self, precision="f64", slices: int = 0, steps=None, energy_out=None) -> dict:
        """Run `steps` (default: every step of the recipe) in order; returns {energy step name: value}."""
        out = {}
        for s in steps if steps is not None else self.w.steps:
            r = self.run_step(s, precision, slices, energy_out)
            if r is not None:
                out[s.name] = r
        return out

    def scheduled(self, precision="f64", slices: int = 0, steps=None, energy_out=None):
        """The recipe's steps (default: all) recorded on a scheduler, which runs them by dependency level:
        the split-precision contractions of a level as one grouped launch.  Energies need ``energy_out``
        (a device double pointer)."""
        T, sch = self.tensors, self.ctx.scheduler()
        for step in steps if steps is not None else self.w.steps:
            if isinstance(step, wl.EnergySpec):
                if energy_out is None:
                    raise ValueError(f"{step.name}: a scheduled energy needs a device result pointer")
                sch.energy_async(step.alpha, T[step.a], step.la, T[step.b], step.lb,
                                 self.energy_slot(step, energy_out))
            elif isinstance(step, wl.AddSpec):
                sch.add(T[step.c], step.lc, step.beta, T[step.a], step.terms)
            elif step.antisym:
                X, lx = self.scratch_for(step)
                sch.contract(step.alpha, X, lx, 0.0, T[step.a], step.la, T[step.b], step.lb, precision, slices)
                sch.add(T[step.c], step.lc, step.beta, X, antisym_terms(step.lc, lx))
            else:
                sch.contract(step.alpha, T[step.c], step.lc, step.beta, T[step.a], step.la, T[step.b], step.lb,
                             precision, slices)
        return sch

    def autotune(self, target: float = 1e-10, steps=None) -> dict:
        """Autotune every contraction step (split precision); later runs with slices = 0 use the choices.

        Tune on the values the steps will see: intermediates written by earlier steps must already hold
        them (run the recipe once first)."""
        T, ctx, out = self.tensors, self.ctx, {}
        for step in steps if steps is not None else self.w.steps:
            if not isinstance(step, wl.ContractSpec):
                continue
            if step.antisym:
                X, lx = self.scratch_for(step)
                out[step.name] = ctx.autotune(X, lx, T[step.a], step.la, T[step.b], step.lb, target)
            else:
                out[step.name] = ctx.autotune(T[step.c], step.lc, T[step.a], step.la, T[step.b], step.lb, target)
        return out

    def run_grouped(self, steps, precision="ozaki_bf16", slices: int = 0) -> None:
        """Independent contraction steps as one contraction group (one grouped GEMM launch), then the
        output antisymmetrisers of those that have one."""
        T, ctx = self.tensors, self.ctx
        after = []
        with ctx.group():
            for step in steps:
                if not isinstance(step, wl.ContractSpec):
                    raise ValueError(f"{step.name}: only contractions can be grouped")
                if step.antisym:
                    X, lx = self.scratch_for(step)
                    ctx.contract(step.alpha, X, lx, 0.0, T[step.a], step.la, T[step.b], step.lb, precision, slices)
                    after.append((step, X, lx))
                else:
                    ctx.contract(step.alpha, T[step.c], step.lc, step.beta, T[step.a], step.la, T[step.b], step.lb,
                                 precision, slices)
        for step, X, lx in after:
            ctx.add(T[step.c], step.lc, step.beta, X, antisym_terms(step.lc, lx))


def build_batch(ctx: Context, sizes, seed: int, scale_tiles: tuple = (20, 40)) -> list:
    """Independent ladder problems R = 1/2 V_vvvv T of the given (O, V) sizes, each with its own tensors
    (seeded per problem index)."""
    out = []
    for k, (o, v) in enumerate(sizes):
        w = wl.ladder_problem(o, v, seed + k, *scale_tiles)
        sp, ts = build(ctx, w)
        out.append((w, Runner(ctx, w, sp, ts)))
    return out
