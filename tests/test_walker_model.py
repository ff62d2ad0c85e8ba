"""CPU model of the edge walker's row search (csrc/dsg_kernels.cuh,
walk_all_entries): every adjacency position must get the row that holds it,
every search must end within its pass bound, and every row start it reads
must lie in [0, n].  The model follows the kernel step by step (a warp of 32
lanes, four positions per lane per step, a 32-row window, then the coarse
sample of 32 row starts S rows apart with S widening by 32 when a pass places
nothing, and a plain binary search after 64 passes) on graphs whose non-empty
rows sit far apart.  No GPU involved."""
import numpy as np
import pytest

U = 4        # positions per lane and step
STEP = 32 * U


def _walk(off, nwarps):
    n = len(off) - 1
    total = int(off[n])
    span = (total + nwarps - 1) // nwarps
    span = 2 * STEP if span < 2 * STEP else (span + STEP - 1) // STEP * STEP
    seen = np.zeros(total, np.int64)
    max_pass = 0

    def rd(i):
        assert 0 <= i <= n, i
        return int(off[i])

    for w in range(nwarps):
        j0 = w * span
        if j0 >= total:
            break
        j1 = min(total, j0 + span)
        lo, hi = 0, n
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if rd(mid) <= j0:
                lo = mid
            else:
                hi = mid
        r = lo
        for jb in range(j0, j1, STEP):
            J = np.arange(jb, jb + STEP).reshape(U, 32).T  # J[lane, t] = jb + lane + 32 t
            valid = J < j1
            owner = np.full(J.shape, r)
            done = ~valid
            win = np.array([rd(min(r + 1 + l, n)) for l in range(32)])
            c = np.searchsorted(win, J, side="right")
            hit = ~done & (c < 32)
            owner[hit] = r + c[hit]
            done |= hit
            b, S, passes = r + 32, 32, 0
            while not done.all():
                if passes == 64:
                    for l, t in zip(*np.nonzero(~done)):
                        lo, hi = b, n
                        while hi - lo > 1:
                            mid = (lo + hi) // 2
                            if rd(mid) <= J[l, t]:
                                lo = mid
                            else:
                                hi = mid
                        owner[l, t] = lo
                    done[:] = True
                    break
                passes += 1
                sample = np.array([rd(b + S * l) if b + S * l < n else rd(n) for l in range(32)])
                placed = 0
                for l, t in zip(*np.nonzero(~done)):
                    j = int(J[l, t])
                    assert rd(b) <= j
                    cnt = int(np.searchsorted(sample, j, side="right"))
                    if cnt < 32:
                        lo, hi = b + S * (cnt - 1), min(b + S * cnt, n)
                        while hi - lo > 1:
                            mid = (lo + hi) // 2
                            if rd(mid) <= j:
                                lo = mid
                            else:
                                hi = mid
                        owner[l, t] = lo
                        done[l, t] = True
                        placed += 1
                b += 31 * S
                if not placed:
                    S *= 32
            max_pass = max(max_pass, passes)
            for l, t in zip(*np.nonzero(valid)):
                v, j = int(owner[l, t]), int(J[l, t])
                assert rd(v) <= j < rd(v + 1), (v, j)
                seen[j] += 1
            if not valid[31, U - 1]:
                break
            r = int(owner[31, U - 1])
    assert (seen == 1).all()
    return max_pass


def _offsets(deg):
    off = np.zeros(len(deg) + 1, np.int64)
    off[1:] = np.cumsum(deg)
    return off


def _cases():
    rng = np.random.default_rng(11)
    pairs_far = np.zeros(70_000, np.int64)
    pairs_far[np.arange(0, 70_000 - 1, 1_100)] = 1
    pairs_far[np.arange(1, 70_000, 1_100)] = 1
    ends = np.zeros(3_000_000, np.int64)
    ends[[0, 1_500_000, 2_999_999]] = [1, 2, 200]
    sparse = (rng.random(3_000) < 0.02) * rng.integers(1, 5, 3_000)
    runs = np.zeros(40_000, np.int64)
    runs[rng.choice(40_000, 60, replace=False)] = rng.integers(1, 200, 60)
    dense = rng.integers(50, 500, 70)
    return [("rows 1,100 apart", pairs_far), ("three rows in 3e6", ends), ("sparse", sparse),
            ("sixty rows in 4e4", runs), ("dense", dense)]


@pytest.mark.parametrize("name,deg", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("nwarps", [1, 3])
def test_every_position_gets_its_row(name, deg, nwarps):
    passes = _walk(_offsets(deg), nwarps)
    assert passes <= 64


def test_far_apart_rows_reach_the_pass_bound():
    # one-entry rows 900 rows apart: a step's 128 positions span ~115,000
    # rows and each pass of 992 rows places only about one of them, so after
    # 64 passes the plain binary search places the rest
    n = 128 * 900 + 10
    deg = np.zeros(n, np.int64)
    deg[np.arange(0, 128 * 900, 900)] = 1
    assert _walk(_offsets(deg), 1) == 64


def test_empty_runs_widen_the_sample():
    # pairs of one-entry rows 1,100 rows apart: the first pass over 992 rows
    # finds nothing, the sample widens to 1,024-row blocks and places the rest
    deg = np.zeros(70_000, np.int64)
    deg[np.arange(0, 70_000 - 1, 1_100)] = 1
    deg[np.arange(1, 70_000, 1_100)] = 1
    assert _walk(_offsets(deg), 1) <= 4
