"""Host-side check of the conv kernel's MMA issue schedule (csrc/qla_conv.cu).

The kernel multiplies each staged input row j of a run by the weights of all
three y taps at once, accumulating into the TMEM blocks of output rows j, j-1,
j-2; output row o (counted over the CTA's runs) owns block (-o) mod NB of a
ring of NB = 512 / NOUT blocks. This test walks the same index arithmetic (run
split, block of a row, valid tap range, split at the ring wrap, accumulation
flag) for the kernel's grids and checks that every output row's block holds
exactly its 9 taps x channel slices when its accumulator is committed, that no
MMA leaves the 512 TMEM columns or the staged weights, that N is a legal MMA
width, and that the barrier phases the epilogue and the MMA warp wait for
match the commit and release counts.
"""
import pytest


def runs(u_begin, u_end, H, TPR):
    u0 = u_begin
    while u0 < u_end:
        y_s = u0 % H
        end = min(u0 - y_s + H, u_end)
        yield end - u0
        u0 = end


def check_cta(CCH, NOUT, H, TPR, u_begin, u_end):
    NB = 512 // NOUT
    blocks, commits = {}, [0] * NB
    g = o = 0
    nmma = 0
    for ln in runs(u_begin, u_end, H, TPR):
        for j in range(ln + 2):
            r, on = g + j, o + j
            b0 = (NB - on % NB) % NB
            if j < ln and on >= NB:  # the MMA warp waits for the epilogue of row on - NB
                assert commits[b0] >= (on - NB) // NB + 1
            k_lo, k_hi = max(0, j - ln + 1), min(2, j)
            wrap = NB - b0
            for kx in range(3):
                for k2 in range(CCH // 2):
                    first = kx == 0 and k2 == 0
                    ka = k_lo
                    while ka <= k_hi:
                        kb = k_hi
                        if ka < wrap <= kb:
                            kb = wrap - 1
                        if first and ka == 0:
                            kb = 0
                        blk = b0 + ka if b0 + ka < NB else b0 + ka - NB
                        n = (kb - ka + 1) * NOUT
                        assert n % 16 == 0 and 16 <= n <= 256
                        assert blk * NOUT + n <= 512
                        b_row = (kx * CCH + 2 * k2) * 3 * NOUT + ka * NOUT
                        assert b_row + 3 * NOUT + n <= 9 * CCH * NOUT  # second 8-channel chunk sits 3 NOUT rows on
                        for ky in range(ka, kb + 1):
                            bb, row = blk + ky - ka, on - ky
                            assert bb < NB and o <= row < o + ln
                            if first and ka == 0:  # accumulation off: the block starts over
                                blocks[bb] = (row, set())
                            owner, terms = blocks[bb]
                            assert owner == row
                            assert (r, ky, kx, k2) not in terms
                            terms.add((r, ky, kx, k2))
                        nmma += 1
                        ka = kb + 1
            if j >= 2:  # acc_full of output row on - 2; the epilogue waits for phase (row / NB) & 1
                od = on - 2
                bd = (NB - od % NB) % NB
                assert commits[bd] == od // NB
                commits[bd] += 1
                owner, terms = blocks[bd]
                i = od - o
                want = {(g + i + ky, ky, kx, k2) for ky in range(3) for kx in range(3) for k2 in range(CCH // 2)}
                assert owner == od and terms == want
        g += ln + 2
        o += ln
    return nmma, o


@pytest.mark.parametrize("CCH,NOUT", [(2, 64), (8, 64), (8, 16)])
@pytest.mark.parametrize("nimg,H,W,grid", [(1, 1024, 1024, 152), (2, 320, 1024, 152), (1, 1, 128, 1), (1, 3, 128, 3),
                                           (3, 5, 256, 7), (1, 70, 128, 1), (1, 300, 128, 2), (4, 512, 256, 152)])
def test_issue_schedule_covers_every_tap_once(CCH, NOUT, nimg, H, W, grid):
    TPR = W // 128
    T = nimg * TPR * H
    total_rows = total_mma = 0
    for cta in range(grid):
        nmma, rows = check_cta(CCH, NOUT, H, TPR, T * cta // grid, T * (cta + 1) // grid)
        total_mma += nmma
        total_rows += rows
    assert total_rows == T
    if H >= 64:  # long runs: well under the 9 x CCH/2 MMAs per output row of one MMA per tap
        assert total_mma / T < 0.6 * 9 * CCH / 2
