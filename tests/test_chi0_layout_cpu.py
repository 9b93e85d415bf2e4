"""Index arithmetic of the chi0 contraction's scratch and slab layouts, restated on the host
(CPU only).

The chi0 epilogue parks each thread's occupied sums in a per-CTA scratch and writes each
frequency's fp32 product into a slab that the frequency reduction reads back with its transpose
(tc_gemm.cuh: park_slot, slab_index; k_tc.cu: chi0_reduce_kernel).  These tests check the
properties the kernels rely on: every slab element has exactly one address inside the slab, a
warp's float4 access covers 512 consecutive bytes in both layouts, and parked slots are distinct
per thread, chunk and part and stay inside the CTA's scratch.
"""
import numpy as np
import pytest


def slab_index(Np, row, col):
    """Element (row, col) of one frequency's slab: 128-row bands stored as [col / 4][row % 128][4]."""
    return (row >> 7) * 128 * Np + (col >> 2) * 512 + (row & 127) * 4 + (col & 3)


def park_slot(cols, cta, lrow, lcol0, part, i):
    """Float offset of chunk i (a multiple of 4) of part `part` for the thread at tile row lrow and
    column half lcol0 / cols: ((part cols / 4 + i / 4) 256 + t) float4s into the CTA's scratch."""
    t = lrow + (lcol0 // cols) * 128
    return cta * 2 * 128 * (2 * cols) + ((part * (cols // 4) + (i >> 2)) * 256 + t) * 4


@pytest.mark.parametrize("Np", [128, 256, 640, 3584])
def test_slab_index_is_a_bijection_onto_the_slab(Np):
    rows, cols = np.meshgrid(np.arange(Np), np.arange(Np), indexing="ij")
    idx = slab_index(Np, rows, cols).ravel()
    assert idx.min() == 0 and idx.max() == Np * Np - 1
    assert np.unique(idx).size == Np * Np


@pytest.mark.parametrize("Np", [128, 3584])
def test_warp_float4_rows_of_the_slab_are_contiguous(Np):
    """32 consecutive rows (a warp, starting at a multiple of 32) storing or loading the float4 of
    columns [4g, 4g + 4): one 512-byte run, each lane's float4 16-byte aligned."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        r0 = int(rng.integers(0, Np // 32)) * 32
        g = int(rng.integers(0, Np // 4))
        starts = np.array([slab_index(Np, r0 + lane, 4 * g) for lane in range(32)])
        assert np.all(starts % 4 == 0)
        assert np.array_equal(starts, starts[0] + 4 * np.arange(32))
        # the float4 itself is the four consecutive columns
        assert all(slab_index(Np, r0, 4 * g + k) == starts[0] + k for k in range(4))


@pytest.mark.parametrize("cols", [32, 64])
def test_parked_slots_are_distinct_and_inside_the_scratch(cols):
    """256 epilogue threads (128 rows x two column halves), two parts, cols / 4 chunks each: the
    slots of one CTA are a permutation of its [2][128][2 cols] floats (in float4 units), and those
    of the next CTA follow."""
    for cta in (0, 3):
        base = cta * 2 * 128 * 2 * cols
        slots = []
        for lrow in range(128):
            for half in range(2):
                for part in range(2):
                    for i in range(0, cols, 4):
                        slots.append(park_slot(cols, cta, lrow, half * cols, part, i))
        slots = np.array(slots)
        assert np.unique(slots).size == slots.size
        assert slots.min() == base and slots.max() == base + 2 * 128 * 2 * cols - 4
        assert np.all((slots - base) % 4 == 0)


@pytest.mark.parametrize("cols", [32, 64])
def test_parked_warp_access_is_one_512_byte_run(cols):
    """A warp's 32 lanes are 32 consecutive tile rows of one column half: for every (part, chunk)
    their float4 slots are consecutive."""
    for w in range(8):   # warps of the 256 epilogue threads: rows 32 (w % 4) .., half w // 4
        lrow0, half = 32 * (w % 4), w // 4
        for part in range(2):
            for i in range(0, cols, 4):
                s = np.array([park_slot(cols, 0, lrow0 + lane, half * cols, part, i) for lane in range(32)])
                assert np.array_equal(s, s[0] + 4 * np.arange(32))
