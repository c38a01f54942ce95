"""Host model of the space-variant kernel's shared-memory layout.

The kernel keeps the four per-term tables of a tile in shared rows: table row
i holds row i of plane 0 at offset 0, of plane 2 at DT, of plane 1 at O1 and
of plane 3 at O1 + DT, with O1 = 16 and the row stride ES = 31 (mod 32).
Steps 1 and 2 give each thread a table line; step 3 reads four corners per own
pixel (nine entries for the hat).  This model restates the geometry and the
thread-to-line mapping and counts, per warp instruction, how many lanes meet
in one 4-byte bank (the number of shared-memory wavefronts it costs)."""
import numpy as np
import pytest

# (RM, T, NTHR, HAT) as instantiated for the launch
GEOMS = [(4, 32, 256, False), (8, 32, 256, False), (16, 64, 512, False),
         (4, 32, 256, True), (8, 32, 256, True)]


def _stride(n, rem):
    while n % 32 != rem:
        n += 1
    return n


def _geom(RM, T, HAT):
    E = T + 2 * RM
    DT = E + (2 if HAT else 1)
    O1 = _stride(2 * DT, 16)
    ES = _stride(O1 + 2 * DT, 31)
    return DT, O1, ES


def _off(q, DT, O1):
    return (O1 if q & 1 else 0) + (q >> 1) * DT


def _lines(E, NTHR):
    """(plane, line) of each thread in step 2 (and, for the box, step 1 with
    (pair, half) in place of the plane), None for idle threads."""
    F = E // 32 * 32
    RMD = E - F
    PW = 2 if RMD <= 16 else 1
    out = []
    for tid in range(NTHR):
        if tid < 4 * F:
            out.append((tid // F, tid % F))
            continue
        i = tid - 4 * F
        w, u = i >> 5, i & 31
        v = u // max(RMD, 1)
        q = w * PW + v
        ok = RMD > 0 and v < PW and q < 4
        out.append((q, F + u - v * RMD) if ok else None)
    return out


def _lines_hat_step1(E, NTHR):
    F = E // 32 * 32
    RMD = E - F
    out = []
    for tid in range(NTHR):
        if tid < 2 * F:
            out.append((tid // F, tid % F))
            continue
        i = tid - 2 * F
        if RMD > 16:
            w, u = i >> 5, i & 31
            out.append((w, F + u) if (w < 2 and u < RMD) else None)
        else:
            p1 = i // max(RMD, 1)
            ok = RMD > 0 and p1 < 2
            out.append((p1, F + i - p1 * RMD) if ok else None)
    return out


def _degree(addrs):
    """Wavefronts of one warp instruction: the largest number of distinct
    addresses that fall into one bank (equal addresses are a broadcast)."""
    by_bank = {}
    for a in addrs:
        by_bank.setdefault(a % 32, set()).add(a)
    return max((len(s) for s in by_bank.values()), default=0)


def _warps(items, NTHR):
    for w in range(NTHR // 32):
        lanes = [x for x in items[32 * w:32 * (w + 1)] if x is not None]
        if lanes:
            yield lanes


@pytest.mark.parametrize("RM,T,NTHR,HAT", GEOMS)
def test_table_lines_are_free_of_bank_conflicts(RM, T, NTHR, HAT):
    DT, O1, ES = _geom(RM, T, HAT)
    assert ES % 2 == 1 and O1 % 32 == 16 and O1 >= 2 * DT
    for R in range(RM + 1):
        E = T + 2 * R
        SL = (E + 1) // 2
        lines = _lines(E, NTHR)
        assert sum(x is not None for x in lines) == 4 * E
        assert sorted(x for x in lines if x) == [(q, l) for q in range(4) for l in range(E)]
        for lanes in _warps(lines, NTHR):
            # step 2: column l of plane q, one row after another
            assert _degree([_off(q, DT, O1) + ES + l + 1 for q, l in lanes]) == 1
            if not HAT:
                # step 1 (box): row l of pair q & 1, half q >> 1, both planes of
                # the pair, at the half's first column (all lanes in step)
                for second in (0, DT):
                    a = [_off(q & 1, DT, O1) + second + (l + 1) * ES + 1 + (q >> 1) * SL
                         for q, l in lanes]
                    assert _degree(a) == 1
        if HAT:
            for lanes in _warps(_lines_hat_step1(E, NTHR), NTHR):
                for second in (0, DT):
                    a = [_off(p, DT, O1) + second + (l + 2) * ES for p, l in lanes]
                    assert _degree(a) == 1


@pytest.mark.parametrize("RM,T,NTHR,HAT", [g for g in GEOMS if not g[3]])
def test_box_corners_of_lanes_with_different_radii(RM, T, NTHR, HAT):
    """A warp's lanes are 32 consecutive own pixels of one tile row.  The
    corners (-r, -r) and (r + 1, r + 1) sit in the bank of the lane's own
    pixel whatever its radius; the other two move by 2r + 1, so a warp whose
    radii step by one costs at most two wavefronts there."""
    DT, O1, ES = _geom(RM, T, HAT)
    rng = np.random.default_rng(0)
    R = RM
    for trial in range(200):
        pi = int(rng.integers(0, T))
        j0 = int(rng.integers(0, T // 32)) * 32
        r0 = int(rng.integers(0, RM))
        cut = int(rng.integers(0, 33))
        rad = [r0 if k < cut else r0 + 1 for k in range(32)]
        if trial % 2:
            rad = rad[::-1]
        for t in range(4):
            o = _off(t, DT, O1)
            c00 = [o + (R + pi - r) * ES + R + j0 + k - r for k, r in enumerate(rad)]
            c11 = [o + (R + pi + r + 1) * ES + R + j0 + k + r + 1 for k, r in enumerate(rad)]
            c01 = [o + (R + pi - r) * ES + R + j0 + k + r + 1 for k, r in enumerate(rad)]
            c10 = [o + (R + pi + r + 1) * ES + R + j0 + k - r for k, r in enumerate(rad)]
            assert _degree(c00) == 1 and _degree(c11) == 1
            assert _degree(c01) <= 2 and _degree(c10) <= 2


@pytest.mark.parametrize("RM,T,NTHR,HAT", GEOMS)
def test_layout_fits_the_blocks_per_sm(RM, T, NTHR, HAT):
    """Tables plus the f~ tile plus the static arrays within the 227 KB a block
    may use, and four blocks per SM (228 KB, 1 KB reserved per block) for the
    256-thread instantiations."""
    DT, O1, ES = _geom(RM, T, HAT)
    E = T + 2 * RM
    dyn = 4 * DT * ES + 4 * E * (E + 1)
    static = 4 * (5 * _stride(E, 16) + 8) if not HAT else 4
    total = dyn + static + 8 * (NTHR // 32) + 4 * (NTHR // 32)
    assert total <= 227 * 1024
    if NTHR == 256:
        assert 4 * (total + 1024) <= 228 * 1024
