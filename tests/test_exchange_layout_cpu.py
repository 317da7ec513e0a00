"""The line DFT's exchange matrix (Line<P, Q, T> in csrc/dos_fft.cuh): entry
(q, k1) lives at q * RP + k1 in the normal layout and at k1 * RP + q in the
transposed one (RP = P + 1 for even P).  Step 1 of thread t writes the entries
of its sub-DFTs q = t + T j; step 2 of thread t reads the entries of its
columns k1 = t + T j.  The bulk passes drop the barrier between two line DFTs
when the second writes in the other layout, which is safe exactly when every
thread then overwrites only entries it read itself: these tests check that
property for the square lines the kernels use it on, and that it fails for the
non-square ones, where the kernels keep the barrier."""
import pytest

LINES = {16: (4, 4, 4), 32: (4, 8, 4), 64: (8, 8, 8), 128: (8, 16, 8), 200: (10, 20, 10),
         256: (16, 16, 16), 400: (20, 20, 20), 512: (16, 32, 16)}


def rp(P):
    return P + 1 if P % 2 == 0 else P


def step1_writes(P, Q, T, t, tr):
    R = rp(P)
    out = set()
    for j in range(Q // T):
        q = t + T * j
        for k1 in range(P):
            out.add(k1 * R + q if tr else q * R + k1)
    return out


def step2_reads(P, Q, T, t, tr):
    R = rp(P)
    out = set()
    for j in range(P // T):
        k1 = t + T * j
        for q in range(Q):
            out.add(k1 * R + q if tr else q * R + k1)
    return out


def thread_private(P, Q, T, first_tr):
    """Second DFT (other layout) writes only what the same thread read in the
    first DFT's step 2, for every thread."""
    return all(step1_writes(P, Q, T, t, not first_tr) <= step2_reads(P, Q, T, t, first_tr)
               for t in range(T))


@pytest.mark.parametrize("m", [16, 64, 256, 400])
def test_square_lines_alternating_layouts_are_thread_private(m):
    P, Q, T = LINES[m]
    assert P == Q == T
    assert thread_private(P, Q, T, first_tr=False)   # normal then transposed
    assert thread_private(P, Q, T, first_tr=True)    # transposed then normal
    # and the transposed layout fits in the exchange buffer of Q * RP entries
    assert max(max(step1_writes(P, Q, T, t, True)) for t in range(T)) < Q * rp(P)


@pytest.mark.parametrize("m", [32, 128, 200, 512])
def test_non_square_lines_need_the_barrier(m):
    P, Q, T = LINES[m]
    assert not (P == Q == T)
    assert not thread_private(P, Q, T, first_tr=False)


@pytest.mark.parametrize("m", sorted(LINES))
def test_each_step_covers_the_matrix_once(m):
    """Step 1 over all threads writes every entry exactly once, step 2 reads
    every entry exactly once, in the normal layout and (square lines, the only
    ones that use it) in the transposed one."""
    P, Q, T = LINES[m]
    for tr in ((False, True) if P == Q == T else (False,)):
        w = [step1_writes(P, Q, T, t, tr) for t in range(T)]
        r = [step2_reads(P, Q, T, t, tr) for t in range(T)]
        assert sum(map(len, w)) == P * Q == len(set().union(*w))
        assert sum(map(len, r)) == P * Q == len(set().union(*r))
        assert set().union(*w) == set().union(*r)


def test_table_matches_the_compiled_line_shapes():
    import glob
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    found = {}
    for f in glob.glob(os.path.join(root, "paper_2604_02624_gb300", "csrc", "pass_m*.cu")):
        for m, p, q, t in re.findall(r"DOS_DEFINE_PASS_OPS\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),", open(f).read()):
            found[int(m)] = (int(p), int(q), int(t))
    assert found == LINES


@pytest.mark.parametrize("m", sorted(LINES))
def test_field_half_is_the_first_half_of_every_sub_dft(m):
    """The halved (N <= M/2) line DFTs: thread t holds position t + T i in
    r[i]; in step 1 the input pp of sub-DFT j is r[j + (Q/T) pp], in step 2
    the output k2 of column k1 = t + T j lands in r[j + (P/T) k2] at position
    k1 + P k2.  Positions below M/2 (the field half) are exactly i < E/2, the
    first P/2 inputs of each first-step sub-DFT and the first Q/2 outputs of
    each second-step one, for every thread."""
    P, Q, T = LINES[m]
    M, E = P * Q, P * Q // T
    QJ, PJ = Q // T, P // T
    for t in range(T):
        for j in range(QJ):
            for pp in range(P):
                i = j + QJ * pp
                x = t + T * i
                assert (x < M // 2) == (pp < P // 2) == (i < E // 2)
        for j in range(PJ):
            k1 = t + T * j
            for k2 in range(Q):
                i = j + PJ * k2
                assert t + T * i == k1 + P * k2
                assert (k1 + P * k2 < M // 2) == (k2 < Q // 2) == (i < E // 2)
