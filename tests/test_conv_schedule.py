"""Host-side check of the conv kernel's MMA issue schedule (csrc/qla_conv.cu).

The kernel multiplies each staged input row j of a run by the weights of all
three y taps at once, accumulating into the TMEM blocks of output rows j, j-1,
j-2; output row o (counted over the CTA's runs) owns block (-o) mod NB of a
ring of NB = 512 / NOUT blocks. The schedule (the run walk, the block of a
row, the valid tap range, the split at the ring wrap, the accumulation flag,
the operand offsets, the accumulator waits and commits) lives in host/device
helpers that the kernel's MMA warp calls; qla_conv_schedule runs the same
helpers on the host and returns what the warp would issue. This test walks
that enumeration for the kernel's grids and checks that every output row's
block holds exactly its 9 taps x channel slices when its accumulator is
committed, that no MMA leaves the 512 TMEM columns, its ring slot or the
staged weights, that N is a legal MMA width, and that the barrier phases the
epilogue and the MMA warp wait for match the commit and release counts.
No GPU is touched.
"""
import pytest

from paper_2301_13601_gb300 import surrogate as S

NS = {(2, 64): 8, (8, 64): 8, (8, 16): 6}  # ring slots of ConvLayout
HP = 130  # staged pixels per ring row (128 + the two halo pixels)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def check_cta(CCH, NOUT, nimg, H, W, grid, cta):
    NB = 512 // NOUT
    ns = NS[(CCH, NOUT)]
    rec = S.conv_schedule(8 * CCH, NOUT, nimg, H, W, grid, cta)
    blocks, commits = {}, [0] * NB
    nmma, rows, released, runs = 0, 0, 0, 0
    for t, r, on, j, ln, a, b, c, d, e, f, g, h, _ in rec.tolist():
        g_run, o_run = r - j, on - j  # ring row and output row where the run starts
        if t == 2:  # the MMA warp waits for the epilogue of the block's previous output row
            assert j < ln and on >= NB and a == (NB - on % NB) % NB
            assert b == ((on // NB) + 1) & 1
            assert commits[a] >= (on - NB) // NB + 1
        elif t == 0:
            kx, k2, ka, kb, blk, acc, a_off, b_off = a, b, c, d, e, f, g, h
            assert 0 <= kx < 3 and 0 <= k2 < CCH // 2 and 0 <= ka <= kb <= 2
            assert max(0, j - ln + 1) <= ka and kb <= min(2, j)  # output rows inside the run
            n = (kb - ka + 1) * NOUT
            assert n % 16 == 0 and 16 <= n <= 256
            assert blk * NOUT + n <= 512
            assert blk == (NB - on % NB + ka) % NB
            # A: 128 pixel rows of 16 B from the slot, the second 8-channel chunk one chunk plane on
            assert a_off == 2 * k2 * ns * HP + kx and kx + 127 < HP
            assert a_off + ns * HP + 127 < CCH * ns * HP
            # B: n rows at [kx][chunk][ky][n], the second chunk 3 NOUT rows on
            assert b_off == (kx * CCH + 2 * k2) * 3 * NOUT + ka * NOUT
            assert b_off + 3 * NOUT + n <= 9 * CCH * NOUT
            first = kx == 0 and k2 == 0 and ka == 0
            assert acc == (0 if first else 1)
            if first:
                assert kb == ka  # the accumulator is started by one MMA alone
            for ky in range(ka, kb + 1):
                bb, row = blk + ky - ka, on - ky
                assert bb < NB and o_run <= row < o_run + ln
                if first:  # accumulation off: the block starts over
                    blocks[bb] = (row, set())
                owner, terms = blocks[bb]
                assert owner == row
                assert (r, ky, kx, k2) not in terms
                terms.add((r, ky, kx, k2))
            nmma += 1
        elif t == 3:  # the tensor cores release the row's ring slot
            assert a == r % ns
            released += 1
            runs += j == 0
        elif t == 1:  # acc_full of output row on - 2; the epilogue waits for phase (row / NB) & 1
            od = on - 2
            assert j >= 2 and a == (NB - od % NB) % NB
            assert commits[a] == od // NB
            commits[a] += 1
            owner, terms = blocks[a]
            want = {(r - 2 + ky, ky, kx, k2) for ky in range(3) for kx in range(3) for k2 in range(CCH // 2)}
            assert owner == od and terms == want
            rows += 1
        else:
            raise AssertionError(f"unknown record type {t}")
        assert g_run >= 0 and o_run >= 0
    assert released == rows + 2 * runs  # every input row once: the run's output rows and its two halo rows
    return nmma, rows


@pytest.mark.parametrize("CCH,NOUT", [(2, 64), (8, 64), (8, 16)])
@pytest.mark.parametrize("nimg,H,W,grid", [(1, 1024, 1024, 152), (2, 320, 1024, 152), (1, 1, 128, 1), (1, 3, 128, 3),
                                           (3, 5, 256, 7), (1, 70, 128, 1), (1, 300, 128, 2), (4, 512, 256, 152)])
def test_issue_schedule_covers_every_tap_once(CCH, NOUT, nimg, H, W, grid):
    TPR = W // 128
    T = nimg * TPR * H
    total_rows = total_mma = 0
    for cta in range(grid):
        nmma, rows = check_cta(CCH, NOUT, nimg, H, W, grid, cta)
        total_mma += nmma
        total_rows += rows
    assert total_rows == T
    if H >= 64:  # long runs: well under the 9 x CCH/2 MMAs per output row of one MMA per tap
        assert total_mma / T < 0.6 * 9 * CCH / 2


def test_schedule_rejects_bad_arguments():
    with pytest.raises(ValueError):
        S.conv_schedule(32, 64, 1, 8, 128, 1, 0)  # unsupported channel pair
    with pytest.raises(ValueError):
        S.conv_schedule(64, 64, 1, 8, 100, 1, 0)  # W not a multiple of 128
    with pytest.raises(ValueError):
        S.conv_schedule(64, 64, 1, 8, 128, 2, 2)  # CTA out of range
