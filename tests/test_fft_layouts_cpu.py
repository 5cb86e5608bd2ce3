"""Index algebra of the warp-per-pencil x transform (fft_pencil_warp in csrc/lpp_fft_dev.cuh),
restated in numpy: the three passes with their intermediate row layouts reproduce the DFT,
every pass writes each row exactly once, and the 16 lanes of every half-warp touch 16
different bank pairs in each shared-memory access (tile rows of LD = 17 complex words,
64-bit accesses: bank pair = (row * LD + column) mod 16)."""
import numpy as np
import pytest

LD = 17


def rows_pass1_write(m, k0):
    return 64 * k0 + ((m + 8 * k0) & 63)


def rows_pass2_write(n0, k0, k1, r1):
    q = 8 * r1
    return q * n0 + ((k0 + r1 * k1 + 2 * n0) & (q - 1))


def pencil_fft(x, sign=-1):
    """The three passes of fft_pencil_warp on one pencil, through a row buffer."""
    n = x.size
    r1 = n // 64
    w = np.exp(sign * 2j * np.pi * np.arange(n) / n)
    buf = np.full(n, np.nan + 0j)
    written = np.zeros(n, int)
    # pass 1: DFT_R1 over n2 of x[m + 64 n2], times w^(m k0)
    for m in range(64):
        v = np.array([x[m + 64 * n2] for n2 in range(r1)])
        y = np.array([np.sum(v * np.exp(sign * 2j * np.pi * np.arange(r1) * k0 / r1)) for k0 in range(r1)])
        for k0 in range(r1):
            row = rows_pass1_write(m, k0)
            buf[row] = y[k0] * w[m * k0]
            written[row] += 1
    assert np.all(written == 1)
    # pass 2: DFT_8 over n1 of y1[n0 + 8 n1, k0], times w^(R1 n0 k1)
    buf2 = np.full(n, np.nan + 0j)
    written[:] = 0
    for n0 in range(8):
        for k0 in range(r1):
            v = np.array([buf[rows_pass1_write(n0 + 8 * n1, k0)] for n1 in range(8)])
            y = np.array([np.sum(v * np.exp(sign * 2j * np.pi * np.arange(8) * k1 / 8)) for k1 in range(8)])
            for k1 in range(8):
                row = rows_pass2_write(n0, k0, k1, r1)
                buf2[row] = y[k1] * w[r1 * n0 * k1]
                written[row] += 1
    assert np.all(written == 1)
    # pass 3: DFT_8 over n0 of y2[n0, q]; X[q + 8 R1 k2]
    out = np.zeros(n, complex)
    q_n = 8 * r1
    for q in range(q_n):
        k0, k1 = q % r1, q // r1
        v = np.array([buf2[rows_pass2_write(n0, k0, k1, r1)] for n0 in range(8)])
        for k2 in range(8):
            out[q + q_n * k2] = np.sum(v * np.exp(sign * 2j * np.pi * np.arange(8) * k2 / 8))
    return out


@pytest.mark.parametrize("n", [256, 512])
def test_three_passes_are_the_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(pencil_fft(x), np.fft.fft(x), rtol=0, atol=1e-9 * np.abs(x).sum())
    np.testing.assert_allclose(pencil_fft(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-9 * np.abs(x).sum())


def _conflict_free(rows, col):
    banks = [(r * LD + col) % 16 for r in rows]
    return len(set(banks)) == len(banks)


@pytest.mark.parametrize("n", [256, 512])
@pytest.mark.parametrize("col", [0, 5, 15])
def test_every_half_warp_access_hits_sixteen_bank_pairs(n, col):
    r1 = n // 64
    q_n = 8 * r1
    lanes_sets = [list(range(h * 16, h * 16 + 16)) for h in range(2)]
    for lanes in lanes_sets:
        for b in range(2):                      # pass 1: butterflies m = lane + 32 b
            ms = [lane + 32 * b for lane in lanes]
            for n2 in range(r1):                # reads of x[m + 64 n2]
                assert _conflict_free([m + 64 * n2 for m in ms], col)
            for k0 in range(r1):                # writes of y1
                assert _conflict_free([rows_pass1_write(m, k0) for m in ms], col)
        for b in range(r1 // 4):                # passes 2 and 3: lane + 32 b
            m2 = [lane + 32 * b for lane in lanes]
            for n1 in range(8):                 # pass-2 reads of y1[n0 + 8 n1, k0]
                assert _conflict_free([rows_pass1_write((v & 7) + 8 * n1, v >> 3) for v in m2], col)
            for k1 in range(8):                 # pass-2 writes of y2
                assert _conflict_free([rows_pass2_write(v & 7, v >> 3, k1, r1) for v in m2], col)
            for n0 in range(8):                 # pass-3 reads of y2[n0, q]
                assert _conflict_free([q_n * n0 + ((q + 2 * n0) & (q_n - 1)) for q in m2], col)
