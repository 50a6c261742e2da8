"""Index permutation of row-major tensors (oracle; test infrastructure only).

Definition (Methods, "Cache-efficient index permutations"): tensors are stored
row-major; permuting the indexes reorders the entries in memory.  With
out axis i = in axis perm[i], out[j_0, ..., j_{r-1}] = in[i] where
i_{perm[a]} = j_a.  `permute` is that definition (numpy.transpose + copy).

`apply_move` / `lr_decompose` restate the paper's left/right moves:
split the indexes into a left group and a right group of gamma indexes; a left
move L-gamma permutes only left indexes (each contiguous block of the right
group's d_gamma entries moves as a whole), a right move R-gamma permutes only
the right group (within each contiguous chunk of d_gamma entries).  Any
permutation decomposes as L-mu, R-nu, L-mu when the middle group (nu - mu
indexes) is at least as large as the right group (mu indexes).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def permute(x: np.ndarray, perm: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.transpose(x, tuple(perm)))


def apply_move(x: np.ndarray, order: Sequence[str], new_order: Sequence[str],
               kind: str, gamma: int) -> np.ndarray:
    """Apply an L-gamma or R-gamma move taking index labels `order` to `new_order`.

    Raises ValueError if the move is not of the stated kind.
    """
    order, new_order = list(order), list(new_order)
    n = len(order)
    if sorted(order) != sorted(new_order):
        raise ValueError("not a permutation")
    if kind == "L":
        if order[n - gamma:] != new_order[n - gamma:]:
            raise ValueError("an L move must keep the right group in place")
        left = n - gamma
        shp = x.shape
        blocks = x.reshape(shp[:left] + (-1,))
        p = [order.index(l) for l in new_order[:left]] + [left]
        out = np.transpose(blocks, p)
        return np.ascontiguousarray(out).reshape([shp[order.index(l)] for l in new_order])
    if kind == "R":
        left = n - gamma
        if order[:left] != new_order[:left]:
            raise ValueError("an R move must keep the left group in place")
        shp = x.shape
        chunks = x.reshape((-1,) + shp[left:])
        p = [0] + [1 + order[left:].index(l) for l in new_order[left:]]
        out = np.transpose(chunks, p)
        return np.ascontiguousarray(out).reshape([shp[order.index(l)] for l in new_order])
    raise ValueError(kind)


def lr_decompose(order: Sequence[str], target: Sequence[str], mu: int, nu: int
                 ) -> List[Tuple[str, int, List[str]]]:
    """Three moves (L-mu, R-nu, L-mu) taking `order` to `target`.

    1. L-mu: indexes that must end in the rightmost mu positions and sit in
       the left/middle groups are moved into the middle group;
    2. R-nu: the rightmost mu indexes are put in their final places;
    3. L-mu: the remaining indexes are put in their final places.
    Requires nu - mu >= mu (middle group at least as large as the right group).
    """
    order, target = list(order), list(target)
    n = len(order)
    if nu - mu < mu or nu > n:
        raise ValueError("need a middle group at least as large as the right group")
    right_final = target[n - mu:]
    lm = order[:n - mu]
    to_right = [l for l in lm if l in right_final]
    others = [l for l in lm if l not in right_final]
    mid_size = nu - mu
    n_left = n - nu
    # keep the leftmost `n_left` others on the left, the rest fill the middle
    step1 = others[:n_left] + to_right + others[n_left:] + order[n - mu:]
    assert len(step1) == n
    tail = step1[n - nu:]
    mid_rest = [l for l in tail if l not in right_final]
    step2 = step1[:n - nu] + mid_rest + right_final
    step3 = list(target)
    return [("L", mu, step1), ("R", nu, step2), ("L", mu, step3)]


def permute_lr(x: np.ndarray, order: Sequence[str], target: Sequence[str],
               mu: int, nu: int) -> np.ndarray:
    cur = list(order)
    for kind, gamma, new in lr_decompose(order, target, mu, nu):
        x = apply_move(x, cur, new, kind, gamma)
        cur = new
    return x
