"""The planner's column-walk unit tables against the lattice's geometry (CPU).

Each unit (column col = x/2 + (L/2) y, segment g of L/K planes) tells a thread
the half index of its first site, the half index of that site's -z
neighbour, the +-y offsets, the x parity of the first site and the two x
offsets the walk alternates between.  This test decodes every unit the way
the walk does and compares each site's index and neighbours with the simple
cubic lattice's definition (periodic, site i = x + L(y + Lz), colour
(x + y + z) mod 2, half index i >> 1), for every even L the shared-memory
kernels take and the thread counts the planner can choose.  The table is
made by host code (csrc/common.cuh) compiled here for the CPU.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1305_6758_gb300", "csrc")


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is needed to compile the planner's host code")
    exe = str(tmp_path_factory.mktemp("units") / "units_dump")
    src = os.path.join(ROOT, "tests", "units_dump.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, src, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    plans = []
    for line in out.splitlines():
        v = [int(t) for t in line.split()]
        L, mixed, tp, U, K = v[:5]
        units = [tuple(v[5 + 4 * u:9 + 4 * u]) for u in range((len(v) - 5) // 4)]
        plans.append((L, mixed, tp, U, K, units))
    return plans


def half(L, x, y, z):
    return ((x % L) + L * ((y % L) + L * (z % L))) >> 1


def sbyte(v):
    v &= 0xFF
    return v - 256 if v >= 128 else v


def test_segments_and_chunks(dump):
    for L, mixed, tp, U, K, units in dump:
        assert L % U == 0 and L % K == 0 and (L // K) % U == 0, (L, U, K)
        assert len(units) == L * L // 2 * K
        # K spreads the units most evenly: no other admissible divisor fills more lanes
        def fill(k):
            n = L * L // 2 * k
            return n / (-(-n // tp) * tp)
        best = max(fill(k) for k in range(1, L + 1) if L % k == 0 and (L // k) % U == 0)
        assert abs(fill(K) - best) < 1e-12


def test_every_unit_matches_the_lattice(dump):
    for L, mixed, tp, U, K, units in dump:
        HL, HP, seg = L // 2, L * L // 2, L // K
        for u, (dx, dy, dz, dw) in enumerate(units):
            g, col = divmod(u, HP)
            hx, y = col % HL, col // HL
            z0 = g * seg
            hh0 = dx & 0x7FFFFFFF
            pa0 = (dx >> 31) & 1 if dx >= 0 else 1
            mz = dy & 0xFFFF
            oxa, oxb = sbyte(dy >> 16), sbyte(dy >> 24)
            oyp, oym = dz, dw
            for c in (0, 1):
                # colour 1 flips the parity and swaps the x offsets
                a, b = (oxa, oxb) if c == 0 else (oxb, oxa)
                for k in range(seg):
                    z = z0 + k
                    # within a chunk the walk alternates (pa, a), (pb, b); an odd
                    # chunk swaps the pairs for the next, so the choice follows k
                    p = (pa0 ^ c ^ (k & 1))
                    ox = a if (k % 2 == 0) else b
                    hh = hh0 + k * HP
                    x = 2 * hx + p
                    assert (x + y + z) % 2 == c
                    assert 2 * hh + p == x + L * (y + L * z), (L, K, u, c, k)
                    # x neighbours: one at the site's own half index, the other at hh + ox
                    assert sorted([hh, hh + ox]) == sorted([half(L, x + 1, y, z), half(L, x - 1, y, z)])
                    assert hh + oyp == half(L, x, y + 1, z)
                    assert hh + oym == half(L, x, y - 1, z)
                    if k == 0:
                        assert mz == half(L, x, y, z - 1)
