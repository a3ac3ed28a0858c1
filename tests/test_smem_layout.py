"""Shared-memory bank model of the one-CTA-per-tile axis-pass kernel.

The kernel stages a tile of G lines of length L in shared memory and touches
it in four patterns: the tile load and store and the potential and kinetic
loops walk it in global-address order (Wi lines of consecutive addresses
side by side), and each Stockham stage reads 8 values per thread at stride
L/R and writes them back at stride Ls.  The hardware serves a warp-wide
access of 8-byte elements in two phases of 16 threads and of 16-byte
elements in four phases of 8 threads; within a phase, threads that touch
different 4-byte words of one of the 32 banks are served one after another.

This test restates that model and the layout rule of `tile_layout`
(csrc/axis_pass.cuh: one pad element every 2^plog, line stride
L + L / 2^plog + X) and checks that the rule removes most of the wavefronts
the unpadded layout needs: every case reaches the minimum (FP64, L >= 64) or
stays within 1.3x of it (FP32, L >= 128), against 2-5x unpadded."""
import math

import pytest


def wavefronts(addrs, size):
    tpp = 128 // size
    total = 0
    for ph in range(0, 32, tpp):
        banks = {}
        for a in addrs[ph:ph + tpp]:
            if a is None:
                continue
            for w in range(size // 4):
                word = a // 4 + w
                banks.setdefault(word % 32, set()).add(word // 32)
        total += max((len(v) for v in banks.values()), default=0)
    return total


def plan(L):
    log2L = int(math.log2(L))
    rem = log2L % 3
    stages = [(8 if rem == 0 else (2 if rem == 1 else 4), 1)]
    Ls = stages[0][0]
    for _ in range(log2L // 3 - (1 if rem == 0 else 0)):
        stages.append((8, Ls))
        Ls *= 8
    return stages


def count(L, G, Wi, size, idx):
    """(wavefronts, minimum) over one tile-order sweep and one FFT."""
    nthr = G * (L // 8)
    tile = G * L
    got = ideal = 0

    def run(addr_of):
        nonlocal got, ideal
        for w in range(0, nthr, 32):
            addrs = [addr_of(t) * size if t < nthr and addr_of(t) is not None else None
                     for t in range(w, w + 32)]
            act = sum(a is not None for a in addrs)
            got += wavefronts(addrs, size)
            ideal += max(1, math.ceil(act * size / 128))

    wl, ll = int(math.log2(Wi)), int(math.log2(L))

    def elem(e):
        return ((e >> (wl + ll)) << wl) | (e & (Wi - 1)), (e >> wl) & (L - 1)

    for it in range(0, tile, nthr):
        run(lambda t: idx(*elem(it + t)) if it + t < tile else None)
    for R, Ls in plan(L):
        NB, Q = 8 // R, L // R
        for beta in range(NB):
            for r in range(R):
                run(lambda t: idx(t // (L // 8), (t % (L // 8)) * NB + beta + r * Q))
        for beta in range(NB):
            for r in range(R):
                def wr(t):
                    j = (t % (L // 8)) * NB + beta
                    k = j & (Ls - 1)
                    return idx(t // (L // 8), (j - k) * R + k + r * Ls)
                run(wr)
    return got, ideal


def tile_layout(L, esz, Wi):
    """The rule of csrc/axis_pass.cuh, restated: (line stride, log2 pad spacing)."""
    if esz == 16:
        plog, X = 3, ((8 // Wi if Wi <= 8 else 1) if L >= 64 else 0)
    elif L >= 128:
        plog, X = 4, (16 // Wi if Wi <= 16 else 1)
    else:
        plog, X = 3, 0
    return L + (L >> plog) + X, plog


CASES = [(size, L, Wi) for size in (16, 8) for L in (64, 128, 256, 512, 1024) for Wi in (1, 2, 4, 8)
         if not (size == 8 and L < 128)]


@pytest.mark.parametrize("size,L,Wi", CASES)
def test_padding_reaches_the_bank_minimum(size, L, Wi):
    G = max(Wi, 4 if L <= 256 else 1)
    ls, plog = tile_layout(L, size, Wi)
    padded, ideal = count(L, G, Wi, size, lambda g, n: g * ls + n + (n >> plog))
    plain, _ = count(L, G, Wi, size, lambda g, n: g * L + n)
    bound = 1.0 if size == 16 else 1.3
    assert padded <= bound * ideal, (padded, ideal)
    assert plain >= 2 * ideal  # what the padding removes
