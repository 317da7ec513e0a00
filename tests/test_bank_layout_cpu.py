"""Shared-memory bank mapping of the pass kernels' layouts, on the host.

The layout constants come from the kernels' own headers
(tests/layout_constants_host.cu, compiled by nvcc as host code).  The bank
model: shared memory serves 128 bytes per wavefront (32 banks of 4 bytes); a
warp's 8-byte accesses are served per half-warp (16 lanes, one bank pair per
lane) and its 16-byte accesses per quarter-warp (8 lanes, one bank quad per
lane); lanes that read the same address share it, lanes that touch different
words of one bank pair (quad) take one wavefront each.  A layout is
conflict-free when every half-warp (quarter-warp) takes one wavefront.

These checks pin the layout claims the kernels' comments make: the twiddle
table's pitch (2 mod 4) puts the pair loads of 8 consecutive table rows on 8
distinct bank quads (an even pitch that is a multiple of 4 had put all 8 on
one at M = 512: 8-way conflicts that made the row passes shared-memory-bound);
the bulk column pass's exchange matrices, stage and transfer-table tile are
conflict-free for its thread mapping; the row passes' are for M = 400 and
M = 512."""
import hashlib
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "layout_constants_host.cu")
CSRC = os.path.join(ROOT, "paper_2604_02624_gb300", "csrc")
HDRS = [os.path.join(CSRC, f) for f in ("dos_fft.cuh", "dos_pass.cuh", "dos_pass_bulk.cuh", "dos_internal.h")]
BUILD = os.path.join(ROOT, "tests", "_build")


_NVCC = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
pytestmark = pytest.mark.skipif(_NVCC is None, reason="nvcc not available")


def _constants():
    nvcc = _NVCC
    key = hashlib.sha1(b"".join(open(f, "rb").read() for f in [SRC] + HDRS)).hexdigest()[:16]
    exe = os.path.join(BUILD, f"layout_constants_{key}")
    if not os.path.exists(exe):
        os.makedirs(BUILD, exist_ok=True)
        cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1", "-x", "cu", SRC, "-o", exe + ".tmp"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        assert p.returncode == 0, p.stdout + p.stderr
        os.replace(exe + ".tmp", exe)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    return {d["M"]: d for d in (json.loads(line) for line in out.stdout.splitlines() if line.strip())}


SHAPES = _constants() if _NVCC else {}
BULK_COLUMN_M = [16, 32, 64, 128, 256, 400, 512]  # M % 16 == 0: the sizes the bulk column kernel runs


def wavefronts(addrs, width):
    """addrs: the float2 index each of a warp's 32 lanes accesses (None:
    inactive); width 1 (8-byte accesses) or 2 (16-byte, even index)."""
    group = 16 if width == 1 else 8
    units = 16 if width == 1 else 8
    total = 0
    for s in range(0, 32, group):
        banks = {}
        for a in addrs[s:s + group]:
            if a is None:
                continue
            u = a // width
            banks.setdefault(u % units, set()).add(u)
        total += max((len(v) for v in banks.values()), default=0)
    return total


def ideal(addrs, width):
    """Wavefronts of a conflict-free access: one per half- (quarter-) warp with an active lane."""
    group = 16 if width == 1 else 8
    return sum(1 for s in range(0, 32, group) if any(a is not None for a in addrs[s:s + group]))


# ---------------------------------------------------------------- twiddle table
@pytest.mark.parametrize("m", [16, 32, 64, 128, 200, 256, 400, 512])
def test_twiddle_pitch_puts_consecutive_rows_on_distinct_bank_quads(m):
    c = SHAPES[m]
    P, Q, TWP = c["P"], c["Q"], c["TWP"]
    assert TWP >= P and TWP % 4 == 2 and c["TWS"] == Q * TWP
    span = min(8, Q)
    for q0 in range(Q - span + 1):
        quads = {((q * TWP) // 2) % 8 for q in range(q0, q0 + span)}
        assert len(quads) == span, (m, q0)


def test_an_even_pitch_that_is_a_multiple_of_4_conflicts():
    """The earlier pitch at M = 512 (16): 8 consecutive rows on one bank quad."""
    assert len({((q * 16) // 2) % 8 for q in range(8)}) == 1


# ---------------------------------------------------------------- bulk column pass
def _col_lanes(c, w):
    """(group, line, element owner) of lane 0..31 of warp w of the bulk column block."""
    GT, GW = c["GT"], c["GW"]
    out = []
    for lane in range(32):
        tid = 32 * w + lane
        out.append((tid // GT, tid % GW, (tid % GT) // GW))
    return out


@pytest.mark.parametrize("m", BULK_COLUMN_M)
def test_bulk_column_exchange_stage_and_tile_are_conflict_free(m):
    c = SHAPES[m]
    P, Q, T, ZX, ZLB = c["P"], c["Q"], c["T"], c["ZX"], c["ZLB"]
    assert c["GROUP_BARS"] and c["GT"] % 32 == 0, "a warp belongs to one group"
    assert ZX % 2 == 0 and ZLB % 16 == 2 and ZLB >= Q * ZX
    square = P == Q == T
    M, HP, HB, GW = c["M"], c["HP"], c["HB"], c["GW"]
    E = M // T
    nwarps = 2 * c["GT"] // 32
    for w in range(nwarps):
        L = _col_lanes(c, w)
        z = lambda g, lc: (g * GW + lc) * ZLB
        checks = []
        for j in range(Q // T):
            # step 1, row layout: entries (q, k1), (q, k1 + 1) of sub-DFT q = t + T j as one 16-byte store
            for k0 in range(0, P - 1, 2):
                checks.append(([z(g, lc) + (t + T * j) * ZX + k0 for g, lc, t in L], 2))
            # twiddle pairs of row q (one table for the block: lanes with one t share the address)
            for k0 in range(0, P - 1, 2):
                checks.append(([(t + T * j) * c["TWP"] + k0 for g, lc, t in L], 2))
        for j in range(P // T):
            # step 2, row layout: column k1 = t + T j, 8-byte reads
            for q in range(Q):
                checks.append(([z(g, lc) + q * ZX + t + T * j for g, lc, t in L], 1))
        if square:
            # transposed layout: step 1 writes column q = t, step 2 reads row k1 = t in pairs
            for k1 in range(P):
                checks.append(([z(g, lc) + k1 * ZX + t for g, lc, t in L], 1))
            for q0 in range(0, Q - 1, 2):
                checks.append(([z(g, lc) + t * ZX + q0 for g, lc, t in L], 2))
        for i in range(E // 2):
            # stage: a group's rows of 8 columns, row t + T i at (row) * 8 + line
            checks.append(([g * 100000 + (t + T * i) * GW + lc for g, lc, t in L], 1))
        for i in range(E):
            # transfer-table tile: |kx| - c0 = hc (line lc of group g), |ky| = t + T i or M - t - T i
            rows = [(t + T * i) if i < E // 2 else (M - t - T * i) for g, lc, t in L]
            hcs = [lc if g == 0 else GW - lc for g, lc, t in L]
            if c["STAGE_H"]:
                addrs = [hc * HP + r for hc, r in zip(hcs, rows)]
            else:
                # box 0 or box 1 of the group's tile, chosen per register (its |ky|
                # range over the element owners) as the kernel does
                b1 = GW * HB - (HP - HB)
                box0 = (T * i + T - 1 < HB) if i < E // 2 else (M - T * i < HB)
                addrs = [g * 100000 + (hc - g) * HB + (r if box0 else r + b1)
                         for (g, lc, t), hc, r in zip(L, hcs, rows)]
            checks.append((addrs, 1))
        for addrs, width in checks:
            assert wavefronts(addrs, width) == ideal(addrs, width), (m, w, width, addrs[:16])


# ---------------------------------------------------------------- row passes
@pytest.mark.parametrize("m", [400, 512])
def test_row_pass_exchange_and_stage_are_conflict_free(m):
    c = SHAPES[m]
    P, Q, T, RP, RZL, SR, RL = c["P"], c["Q"], c["T"], c["RP"], c["RZL"], c["SR"], c["RL"]
    square = P == Q == T
    E = c["M"] // T
    nthr = T * RL
    for w in range((nthr + 31) // 32):
        L = [((32 * w + lane) // T, (32 * w + lane) % T) if 32 * w + lane < nthr else None for lane in range(32)]
        checks = []
        for i in range(E):
            checks.append([l * SR + t + T * i if (l, t) != (None, None) else None
                           for l, t in (x or (None, None) for x in L)])
        for j in range(Q // T):
            for k1 in range(P):
                checks.append([x[0] * RZL + (x[1] + T * j) * RP + k1 if x else None for x in L])
                if square:
                    checks.append([x[0] * RZL + k1 * RP + x[1] + T * j if x else None for x in L])
        for j in range(P // T):
            for q in range(Q):
                checks.append([x[0] * RZL + q * RP + x[1] + T * j if x else None for x in L])
                if square:
                    checks.append([x[0] * RZL + (x[1] + T * j) * RP + q if x else None for x in L])
        for addrs in checks:
            assert wavefronts(addrs, 1) == ideal(addrs, 1), (m, w, addrs[:16])


@pytest.mark.parametrize("m", [400, 512])
def test_row_pass_twiddle_pairs_within_a_line_are_conflict_free(m):
    """The row passes' quarter-warps of 8 consecutive element owners of one line
    read 8 consecutive table rows: distinct bank quads.  (A quarter-warp that
    straddles two lines, as at T = 20, may pair two rows on one quad.)"""
    c = SHAPES[m]
    P, Q, T, TWP, RL = c["P"], c["Q"], c["T"], c["TWP"], c["RL"]
    nthr = T * RL
    total, best = 0, 0
    for w in range((nthr + 31) // 32):
        L = [((32 * w + lane) // T, (32 * w + lane) % T) if 32 * w + lane < nthr else None for lane in range(32)]
        for j in range(Q // T):
            for k0 in range(0, P - 1, 2):
                addrs = [(x[1] + T * j) * TWP + k0 if x else None for x in L]
                for s in range(0, 32, 8):
                    quarter = [x for x in L[s:s + 8] if x]
                    if len({l for l, t in quarter}) == 1:  # one line
                        sub = addrs[s:s + 8] + [None] * 24
                        assert wavefronts(sub, 2) == 1, (m, w, s)
                total += wavefronts(addrs, 2)
                best += ideal(addrs, 2)
    assert total <= 1.25 * best, (total, best)
