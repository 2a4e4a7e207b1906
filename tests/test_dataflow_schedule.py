"""Host-side model of the 3-D dataflow normal operator's work list
(c3_dataflow_kernel): the item decode, the dependency waits and the counter
targets, checked for every (ny, nz) the kernel is built for, ragged x
blocks and coil groups, and both item sizes (one or two z planes per A item,
one or two line units per B item).

Blocks claim items in increasing index order, a block holds at most its
current item and the next one it claimed, and every wait is bounded.  The
kernel therefore cannot stall as long as every wait of an item is met by
items of lower index only: the lowest unfinished item then always has its
dependencies done.  The model runs the items in index order and asserts
exactly that, plus that every (phase, coil, plane), (phase, coil, line unit)
and (phase, plane) is covered once, that the counters reach their targets
exactly, and that they fit the buffer the plan allocates."""
import pytest

DN1, DTX = 16, 16
N2_CASES = [(8, 8), (12, 8), (16, 8), (20, 8), (24, 8), (8, 12), (12, 12), (16, 12), (8, 16),
            (12, 16), (16, 16)]


def df_consts(n2y, n2z):
    ny, nz = 16 * n2y, 16 * n2z
    rmax = max(n2y, n2z, DN1)
    lpb = rmax // n2z if (rmax % n2z == 0 and ny % (rmax // n2z) == 0) else 1
    return ny, nz, lpb, ny // lpb


def counter_ints(nx, C, nz, cg):
    nb, ng = -(-nx // DTX), -(-C // cg)
    return nb * ng * (2 * cg + nz) + 2


def run_schedule(nx, n2y, n2z, C, CG, m):
    ny, nz, lpb, nbi = df_consts(n2y, n2z)
    ma = mb = m
    assert nz % ma == 0 and nbi % mb == 0, "item sizes must divide the counter targets"
    nb, ng = -(-nx // DTX), -(-C // CG)
    cg_last = C - (ng - 1) * CG
    NA, NBm = nz // ma, nbi // mb
    per_full = CG * (NA + NBm) + nz
    per_last = cg_last * (NA + NBm) + nz
    per_blk = (ng - 1) * per_full + per_last
    total = nb * per_blk
    P = nb * ng
    # counter layout of the kernel: cntA[P*CG], cntB[P*CG], cntCz[P*nz], next, err
    offA, offB, offC = 0, P * CG, 2 * P * CG
    n_int = offC + P * nz + 2
    assert n_int == counter_ints(nx, C, nz, CG)
    cnt = [0] * n_int
    seenA, seenB, seenC = set(), set(), set()
    for it in range(total):
        b = it // per_blk
        rr = it - b * per_blk
        g = min(rr // per_full, ng - 1)
        rr -= g * per_full
        k = b * ng + g
        cg = cg_last if g == ng - 1 else CG
        if rr < cg * NA:
            c = rr // NA
            z0 = (rr - c * NA) * ma
            for z in range(z0, z0 + ma):
                # the slot (k & 1) plane is free once phase k - 2's C item of
                # that plane ran (it waited for every B item of its phase)
                if k >= 2:
                    assert cnt[offC + (k - 2) * nz + z] >= 1, ("A waits C(k-2)", it)
                key = (k, c, z)
                assert key not in seenA
                seenA.add(key)
            cnt[offA + k * CG + c] += ma
        elif rr < cg * (NA + NBm):
            q = rr - cg * NA
            c = q // NBm
            u0 = (q - c * NBm) * mb
            assert cnt[offA + k * CG + c] >= nz, ("B waits A", it)
            for u in range(u0, u0 + mb):
                key = (k, c, u)
                assert key not in seenB
                seenB.add(key)
            cnt[offB + k * CG + c] += mb
        else:
            z = rr - cg * (NA + NBm)
            assert 0 <= z < nz
            for c in range(cg):
                assert cnt[offB + k * CG + c] >= nbi, ("C waits B", it)
            if g > 0:
                assert cnt[offC + (k - 1) * nz + z] >= 1, ("C waits C(k-1)", it)
            key = (k, z)
            assert key not in seenC
            seenC.add(key)
            cnt[offC + k * nz + z] += 1
    # coverage and exact targets
    for k in range(P):
        cg = cg_last if k % ng == ng - 1 else CG
        for c in range(CG):
            want_a, want_b = (nz, nbi) if c < cg else (0, 0)
            assert cnt[offA + k * CG + c] == want_a and cnt[offB + k * CG + c] == want_b
        assert all(cnt[offC + k * nz + z] == 1 for z in range(nz))
    assert len(seenA) == sum(nz * (cg_last if k % ng == ng - 1 else CG) for k in range(P))
    assert len(seenB) == sum(nbi * (cg_last if k % ng == ng - 1 else CG) for k in range(P))
    assert len(seenC) == P * nz
    # every unit covers lpb ky lines: the B items cover all ny lines of a coil
    assert nbi * lpb == ny
    return total


@pytest.mark.parametrize("n2", N2_CASES, ids=["%dx%d" % (16 * a, 16 * b) for a, b in N2_CASES])
@pytest.mark.parametrize("m", [1, 2])
def test_schedule_is_claim_order_safe(n2, m):
    n2y, n2z = n2
    for nx, C, CG in [(4, 1, 1), (20, 3, 2), (40, 9, 8), (16, 17, 4), (36, 5, 3), (24, 8, 8),
                      (48, 64, 8), (20, 33, 7)]:
        run_schedule(nx, n2y, n2z, C, CG, m)


@pytest.mark.parametrize("m", [1, 2])
def test_full_workload_schedule(m):
    # 256 x 256 x 128, 32 coils in groups of 8 (16 x-blocks x 4 groups)
    total = run_schedule(256, 16, 8, 32, 8, m)
    ny, nz, lpb, nbi = df_consts(16, 8)
    assert total == 16 * 4 * (8 * (nz // m + nbi // m) + nz)
