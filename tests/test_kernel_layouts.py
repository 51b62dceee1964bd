"""Shared-memory index maps of the two-pass plane transforms, restated from
k_fft32_plane.cu and checked on the CPU: every index stays inside the
plane (Nx/2 + 1 rows of pitch (Ny + 1) | 1), the row and pair assignments
cover each row / pair once, the exchange slots of a pair are distinct, and
the accesses of a half-warp (two lane groups of 8) hit distinct banks where
the layout intends it.  A wrong map here is a shared-memory fault on the
GPU (it was one, at Nx = 64), so the check runs before any GPU run."""
import pytest


def _maps(n):
    nx = ny = n
    nxh, nxq, ldp = nx // 2 + 1, nx // 2, (ny + 1) | 1
    YA, YB = 8, n // 8
    return nx, ny, nxh, nxq, ldp, YA, YB


def _slot(a, c, nxq):
    sl = 8 * c + ((a + c) & 7)
    return sl & (nxq - 1), (1 if sl >= nxq else 0)


@pytest.mark.parametrize("n", [64, 128])
def test_two_pass_plane_indices_stay_inside_the_plane(n):
    nx, ny, nxh, nxq, ldp, YA, YB = _maps(n)
    size = nxh * ldp
    rows = sorted(k0 + w + 8 * g for k0 in range(0, nxq, 32) for w in range(8) for g in range(4))
    assert rows == list(range(nxq))
    pairs = sorted(k0 + 16 * (w >> 2) + (w & 3) + 4 * g for k0 in range(0, ny // 2, 32)
                   for w in range(8) for g in range(4))
    assert pairs == list(range(ny // 2))
    ymat = {a * YB + ((a + c) & (YB - 1)) for a in range(YA) for c in range(YB)}
    assert ymat == set(range(YA * YB)) and max(ymat) < ldp and ny <= ldp
    slots = {_slot(a, c, nxq) for a in range(YA) for c in range(YB)}
    assert len(slots) == YA * YB
    for row, col in slots:
        for ca in range(0, ny, 2):
            assert 0 <= row * ldp + ca + col < size
            assert row < nxq                    # the Nyquist row is not part of the matrix


def _worst(addresses):
    banks = {}
    for x in addresses:
        banks[x % 16] = banks.get(x % 16, 0) + 1     # 8-byte words: 16 bank pairs
    return max(banks.values())


@pytest.mark.parametrize("n", [64, 128])
def test_two_pass_plane_half_warps_avoid_bank_conflicts(n):
    nx, ny, nxh, nxq, ldp, YA, YB = _maps(n)
    assert ldp % 16 == 1
    # y: the two rows of a half-warp are 8 apart
    for c in range(YB):
        assert _worst([(r0 + 8 * g) * ldp + a * YB + ((a + c) & (YB - 1)) for g in (0, 1) for a in range(YA)
                       for r0 in (0,)]) == 1
    # x pass 1: the pairs of a half-warp are 4 apart (columns 8 apart)
    for c in range(YB):
        addr = []
        for ca in (0, 8):
            for a in range(YA):
                row, col = _slot(a, c, nxq)
                addr.append(row * ldp + ca + col)
        assert _worst(addr) == 1
    # x Hermitian reads: rows gl + 8 j (and their mirrors) of the pair's column
    for j in range(YB):
        addr = [((gl + 8 * j) if gl + 8 * j <= nxq else nx - gl - 8 * j) * ldp + ca
                for ca in (0, 8) for gl in range(YA)]
        assert _worst(addr) <= 2
