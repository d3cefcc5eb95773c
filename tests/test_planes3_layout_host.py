"""Shared-memory layout and row chunking of the 3D plane-group field kernel
(csrc/march_layout.cuh, csrc/field_tile.cuh Reach), compiled by nvcc and run on
the host.  Checked from the kernel's access pattern, not by retyping offsets:
the staged rows of a stage are disjoint, 16-byte aligned and fill it; every
column the x1 stencils of Faraday (d_E at B columns) and Ampere (d_B at the
strip's E columns) read lies inside its staged region, for every strip width,
tap count and plane count; the default FP32 shape keeps four CTAs per SM; the
automatic row chunk minimises rounds x (rows + 2).  CPU only."""
import math
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2004_03754_gb300", "csrc")
SMEM_PER_SM = 233472        # 228 KB of shared memory per SM
SMEM_PER_CTA_RESERVED = 1024
BAR_BYTES = 128             # the ring's mbarriers, padded


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = str(tmp_path_factory.mktemp("p3") / "planes3_layout_check_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                           "-o", exe, os.path.join(HERE, "native", "planes3_layout_check_host.cu")])
    return exe


def _layouts(harness, reqs):
    """reqs: (V, MT, SW, P, NS) -> list of dicts with the region widths and row offsets."""
    inp = "".join("L %d %d %d %d %d\n" % r for r in reqs)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout
    res, cur = [], None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "L":
            we, wb, de, le, db, lb, stage, warp, cta = map(int, f[1:])
            cur = dict(WE=we, WB=wb, DE=de, LE=le, DB=db, LB=lb, stage=stage, warp=warp, cta=cta,
                       E={}, B={})
            res.append(cur)
        else:
            cur[f[0]][(int(f[1]), int(f[2]))] = int(f[3])
    assert len(res) == len(reqs)
    return res


SHAPES = [(V, MT, SW, P, NS) for V in (4, 2) for MT in (8, 16, 32)
          for SW in ((32, 64, 96, 128, 160, 224) if V == 4 else (16, 32, 64, 96))
          for P in (1, 2, 3, 4, 6, 8) for NS in (2, 3)]


def test_staged_rows_are_disjoint_aligned_and_fill_the_stage(harness):
    for (V, MT, SW, P, NS), L in zip(SHAPES, _layouts(harness, SHAPES)):
        spans = [(o, o + L["WE"]) for o in L["E"].values()] + [(o, o + L["WB"]) for o in L["B"].values()]
        # E: planes k0-1 .. k0+P (three components, two on the top plane); B: B1 B2 of
        # plane k0-1, three components of the P planes
        assert len(L["E"]) == 3 * (P + 1) + 2 and len(L["B"]) == 2 + 3 * P
        spans.sort()
        assert spans[0][0] == 0 and spans[-1][1] == L["stage"], (V, MT, SW, P)
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 == b0, (V, MT, SW, P, a1, b0)          # disjoint and no gap
        for o, _ in spans:
            assert o % V == 0                                # 16-byte bulk-copy destinations
        assert L["stage"] % V == 0 and L["warp"] % V == 0
        # ring of NS stages, per warp B^{n+1/2} row t [3][WB] and row t-1's B1, B3 [2][SW],
        # then plane k0-1's B1, B2 [2][WB]
        assert L["warp"] >= 3 * L["WB"] + 2 * SW
        assert L["cta"] >= NS * L["stage"] + P * L["warp"] + 2 * L["WB"]


def test_stencil_reads_stay_inside_the_staged_regions(harness):
    for (V, MT, SW, P, NS), L in zip(SHAPES, _layouts(harness, SHAPES)):
        WE, WB, DE, LE, DB, LB = (L[k] for k in ("WE", "WB", "DE", "LE", "DB", "LB"))
        e0 = -DB - DE   # first global column of the E region, relative to the strip start i0
        b0 = -DB        # first of the B region
        # Faraday at every B column i of the region, V at a time from a window of LE values
        # starting at the group's first column: d_E reads E at i + m and i - m + 1
        for col in range(0, WB, V):
            assert col + LE <= WE and col + DE + V <= WE
            for v in range(V):
                i = b0 + col + v
                for m in range(1, MT + 1):
                    for x in (i + m, i - m + 1):
                        assert 0 <= x - e0 < WE, (V, MT, SW, col, v, m)
                        # the window index the stencil uses for it
                        assert col <= x - e0 < col + LE
        # Ampere at every strip column i in [0, SW): d_B reads B at i + m - 1 and i - m;
        # E^n at i itself, and the x2 neighbour row at the same B column
        for oc in range(0, SW, V):
            assert oc + LB <= WB and oc + DB + V <= WB and oc + DB + DE + V <= WE
            for v in range(V):
                i = oc + v
                assert 0 <= i - e0 < WE and 0 <= i - b0 < WB
                for m in range(1, MT + 1):
                    for x in (i + m - 1, i - m):
                        assert 0 <= x - b0 < WB, (V, MT, SW, oc, v, m)
                        assert oc <= x - b0 < oc + LB
        # the plane-k0-1 recomputation covers the strip's B columns DB .. DB+SW
        assert DB + SW <= WB
        # one bulk copy per thread: 6P+7 rows on 32P threads
        assert len(L["E"]) + len(L["B"]) <= 32 * P


def test_default_shapes_fit(harness):
    # FP32 fields: 128 columns, 4 planes, 2 stages -> 4 CTAs per SM; FP64 (8-byte values)
    # 64 columns, 4 planes; compensated pairs (8 bytes) 64 columns, 8 planes
    (f32, f64, dfl) = _layouts(harness, [(4, 16, 128, 4, 2), (2, 16, 64, 4, 2), (2, 16, 64, 8, 2)])
    per_cta = lambda L, size: L["cta"] * size + BAR_BYTES + SMEM_PER_CTA_RESERVED
    assert SMEM_PER_SM // per_cta(f32, 4) == 4
    assert f32["WE"] == 192 and f32["WB"] == 160      # E region sw + 64, B region sw + 32 (M = 16)
    for L, size in ((f32, 4), (f64, 8), (dfl, 8)):
        assert L["cta"] * size + BAR_BYTES <= 200 * 1024   # the argument check's limit
        assert SMEM_PER_SM // per_cta(L, size) >= 1


def test_row_chunk_minimises_rounds_times_rows(harness):
    reqs = [(256, 512, 608), (256, 512, 456), (128, 128, 456), (1024, 24, 608), (37, 5, 3),
            (12, 10, 608), (2048, 4, 152), (1, 7, 9), (300, 1, 1)]
    inp = "".join("R %d %d %d\n" % r for r in reqs)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout
    got = [int(l.split()[1]) for l in out.splitlines()]
    for (n2, cols, slots), r in zip(reqs, got):
        assert 1 <= r <= n2
        rounds = lambda rr: math.ceil(cols * math.ceil(n2 / rr) / slots)
        best = min(rounds(math.ceil(n2 / c)) * (math.ceil(n2 / c) + 2)
                   for c in range(1, min(n2, 256) + 1))
        assert rounds(r) * (r + 2) == best, (n2, cols, slots, r)
