"""Tuning search spaces written out by definition — TEST INFRASTRUCTURE.

A space is an ordered list of (parameter, ordered values) pairs.  Its
configurations are the Cartesian product, enumerated with the first parameter
outermost (the order of Table 1); a configuration's *canonical index* is its
position in that full product, before any restriction is applied.  Restrictions
(Sec. 5, "tunable parameter values ... listed in Table 1", plus the limits any
CUDA launch has) remove configurations:

  * threads per block ``block_x * block_y <= 1024``;
  * with shared-memory staging, the halo tile
    ``(block_y*tile_y + fh - 1) * round_up(block_x*tile_x + fw - 1, 4) * 4`` bytes
    must fit the per-block shared-memory limit (232448 bytes on GB300).

Parameter names follow Table 1: block_size_x / block_size_y / tile_size_x /
tile_size_y are spelled block_x / block_y / tile_x / tile_y; ``smem`` is
use_shmem; ``unroll`` is the loop-unrolling switch of Sec. 3.
"""
from __future__ import annotations

import itertools

PARAMS = ("block_x", "block_y", "tile_x", "tile_y", "smem", "unroll")

SPACES = {
    # 4 x 4 x 2 x 2 x 2 x 2 = 256 (the 256-config small workload; unroll is the
    # parameter that brings 128 listed combinations to 256).
    "small": (("block_x", (16, 32, 64, 128)), ("block_y", (1, 2, 4, 8)),
              ("tile_x", (1, 2)), ("tile_y", (1, 2)), ("smem", (0, 1)), ("unroll", (0, 1))),
    # powers of two 16..256 x 1..16, tiles 1..8, smem and unroll on/off.
    "full": (("block_x", (16, 32, 64, 128, 256)), ("block_y", (1, 2, 4, 8, 16)),
             ("tile_x", tuple(range(1, 9))), ("tile_y", tuple(range(1, 9))),
             ("smem", (0, 1)), ("unroll", (0, 1))),
}

SMEM_LIMIT = 232448
MAX_THREADS = 1024


def round_up(v, m):
    return (v + m - 1) // m * m


def smem_bytes(cfg, fw, fh):
    if not cfg["smem"]:
        return 0
    rows = cfg["block_y"] * cfg["tile_y"] + fh - 1
    cols = round_up(cfg["block_x"] * cfg["tile_x"] + fw - 1, 4)
    return rows * cols * 4


def is_valid(cfg, fw, fh, smem_limit=SMEM_LIMIT, max_threads=MAX_THREADS):
    if cfg["block_x"] * cfg["block_y"] > max_threads:
        return False
    return smem_bytes(cfg, fw, fh) <= smem_limit


def enumerate_space(space, fw, fh, smem_limit=SMEM_LIMIT, valid_only=True):
    """[(canonical_index, cfg_dict)] in canonical order."""
    if isinstance(space, str):
        space = SPACES[space]
    names = [n for n, _ in space]
    out = []
    for idx, vals in enumerate(itertools.product(*[v for _, v in space])):
        cfg = dict(zip(names, vals))
        if not valid_only or is_valid(cfg, fw, fh, smem_limit):
            out.append((idx, cfg))
    return out


def neighbours(space, cfg):
    """Configurations that differ from ``cfg`` in exactly one parameter, by one
    step in that parameter's ordered value list (validity not checked)."""
    if isinstance(space, str):
        space = SPACES[space]
    res = []
    for name, vals in space:
        k = vals.index(cfg[name])
        for d in (-1, 1):
            if 0 <= k + d < len(vals):
                c = dict(cfg)
                c[name] = vals[k + d]
                res.append(c)
    return res


def canonical_index(space, cfg):
    if isinstance(space, str):
        space = SPACES[space]
    idx = 0
    for name, vals in space:
        idx = idx * len(vals) + vals.index(cfg[name])
    return idx
