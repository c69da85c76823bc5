"""Conversion between the library's colour-relative table layout (as
documented in include/motif.h) and the oracle's absolute-mask layout."""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def masks_of_size(nbits: int, size: int) -> list[int]:
    return [m for m in range(1 << nbits) if bin(m).count("1") == size]


@lru_cache(maxsize=None)
def c_index_map(k: int, h: int) -> np.ndarray:
    """[c_v, rho] -> rank (among size-h masks of k colours, ascending) of the
    colour set C = {c_v} + (relative set number rho, c_v re-inserted)."""
    rel = masks_of_size(k - 1, h - 1)
    absr = {m: i for i, m in enumerate(masks_of_size(k, h))}
    out = np.zeros((k, len(rel)), np.int64)
    for cv in range(k):
        for rho, r in enumerate(rel):
            low = r & ((1 << cv) - 1)
            C = low | ((r >> cv) << (cv + 1)) | (1 << cv)
            out[cv, rho] = absr[C]
    return out


@lru_cache(maxsize=None)
def s_index_map(k: int, h: int) -> np.ndarray:
    """[c_v, rho] -> rank among size-h masks of the set C'' (without c_v)."""
    rel = masks_of_size(k - 1, h)
    absr = {m: i for i, m in enumerate(masks_of_size(k, h))}
    out = np.zeros((k, len(rel)), np.int64)
    for cv in range(k):
        for rho, r in enumerate(rel):
            low = r & ((1 << cv) - 1)
            out[cv, rho] = absr[low | ((r >> cv) << (cv + 1))]
    return out


def to_u128_pairs(a: np.ndarray) -> np.ndarray:
    """[..., words] uint64 (1 or 2 words) -> [..., 2] (low, high)."""
    if a.shape[-1] == 2:
        return a
    z = np.zeros(a.shape[:-1] + (2,), np.uint64)
    z[..., 0] = a[..., 0]
    return z


def gpu_c_as_oracle(gpu: np.ndarray, colors: np.ndarray, k: int, h: int, r: int) -> np.ndarray:
    """GPU level-h c table [n, Bc*r, words] (set-major: entry (set rho, shape s)
    at rho * r + s) -> oracle layout [n, r, C(k,h), 2]."""
    n = gpu.shape[0]
    Bc = math.comb(k - 1, h - 1)
    g = to_u128_pairs(gpu).reshape(n, Bc, r, 2)               # set-major rows
    out = np.zeros((n, r, math.comb(k, h), 2), np.uint64)
    idx = c_index_map(k, h)[colors.astype(np.int64)]          # [n, Bc]
    rows = np.arange(n)[:, None]
    for s in range(r):
        out[rows, s, idx] = g[:, :, s]
    return out


def gpu_s_as_oracle(gpu: np.ndarray, colors: np.ndarray, k: int, h: int, r: int) -> np.ndarray:
    n = gpu.shape[0]
    Bs = math.comb(k - 1, h)
    g = to_u128_pairs(gpu).reshape(n, Bs, r, 2)               # set-major rows
    out = np.zeros((n, r, math.comb(k, h), 2), np.uint64)
    idx = s_index_map(k, h)[colors.astype(np.int64)]
    rows = np.arange(n)[:, None]
    for s in range(r):
        out[rows, s, idx] = g[:, :, s]
    return out


def neighbor_sums(table: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """S[v] = sum over neighbours u of table[u] for u128 (low, high) pairs,
    exactly (32-bit limbs, carries propagated)."""
    n = row_ptr.shape[0] - 1
    flat = table.reshape(table.shape[0], -1, 2)
    lo = flat[..., 0]
    hi = flat[..., 1]
    limbs = [(lo & 0xFFFFFFFF).astype(np.int64), (lo >> 32).astype(np.int64),
             (hi & 0xFFFFFFFF).astype(np.int64), (hi >> 32).astype(np.int64)]
    deg = np.diff(row_ptr)
    sums = []
    for L in limbs:
        g = L[col.astype(np.int64)]
        s = np.zeros((n,) + L.shape[1:], np.int64)
        nz = deg > 0
        if g.shape[0]:
            red = np.add.reduceat(g, row_ptr[:-1][nz], axis=0)
            s[nz] = red
        sums.append(s)
    out = np.zeros(flat.shape, np.uint64)
    carry = np.zeros(sums[0].shape, np.int64)
    words = []
    for L in sums:
        t = L + carry
        words.append((t & 0xFFFFFFFF).astype(np.uint64))
        carry = t >> 32
    out[..., 0] = words[0] | (words[1] << np.uint64(32))
    out[..., 1] = words[2] | (words[3] << np.uint64(32))
    return out.reshape(table.shape)
