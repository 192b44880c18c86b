"""Helpers shared by GPU parity tests: run a recipe on both sides, compare by block tile tuple."""
import numpy as np

import oracle as O


def gpu_to_oracle_layout(G, R: "O.Tensor") -> np.ndarray:
    """GPU tensor data re-laid in the oracle's block order (matched by tile tuple)."""
    g = G.download()
    out = np.empty(R.n_elems)
    idx = {tuple(t): k for k, t in enumerate(G.block_tiles.tolist())}
    assert G.n_blocks == R.n_blocks
    for b in range(R.n_blocks):
        k = idx[tuple(R.block_tiles[b].tolist())]
        n = (R.block_off[b + 1] if b + 1 < R.n_blocks else R.n_elems) - R.block_off[b]
        out[R.block_off[b]:R.block_off[b] + n] = g[G.block_offsets[k]:G.block_offsets[k] + n]
    return out


def rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (d if d > 0 else 1.0))


def oracle_to_gpu_layout(R: "O.Tensor", values: np.ndarray, G) -> np.ndarray:
    """Oracle-ordered block data re-laid in the GPU tensor's block order (matched by tile tuple)."""
    out = np.zeros(G.n_elems)
    idx = {tuple(t): k for k, t in enumerate(G.block_tiles.tolist())}
    assert G.n_blocks == R.n_blocks
    for b in range(R.n_blocks):
        k = idx[tuple(R.block_tiles[b].tolist())]
        n = (R.block_off[b + 1] if b + 1 < R.n_blocks else R.n_elems) - R.block_off[b]
        out[G.block_offsets[k]:G.block_offsets[k] + n] = values[R.block_off[b]:R.block_off[b] + n]
    return out
