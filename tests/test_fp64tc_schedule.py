"""Host models of the FP64-TC kernels' step schedules (dwt_fp64tc.cu): every
role of a persistent CTA walks the same clusters in its own loop nest, and
they meet only through counted mbarriers, so the loop nests must agree on
the number and order of hand-offs.  These models restate each role's loops
as the kernels run them and check, for every bandwidth up to 512 and the
cluster lists one CTA walks:

* forward: the producers' staged row groups are the converters' groups in
  the same order (and rows); each converter step signals one `ready` that
  the issuer consumes with one MMA batch into the step's tile accumulator
  (at most four tiles per pass, TMEM columns 128 t); a chunk's data operand
  is cut once per pass, before the pass's first tile of that chunk;
* inverse: per tile slot, producer ring groups equal converter ring groups;
  afull / mdone completions per tile slot equal the issuer's waits; a tile
  slot whose first sample lies past 2B is skipped by all three roles.
"""
import math

import pytest

KC_FWD, TM_FWD, G_FWD = 128, 64, 16
KC_INV, TM_INV = 32, 128


def clusters_of_cta(B, cta, grid):
    """Representatives m of the clusters CTA `cta` walks (only l0 = m matters here)."""
    reps = [(m, mp) for m in range(B) for mp in range(m + 1)]
    return [reps[i][0] for i in range(cta, len(reps), grid)]


# ---- forward -------------------------------------------------------------------
def fwd_producer(B, l0s):
    n = 2 * B
    nchunks = math.ceil(n / KC_FWD)
    for l0 in l0s:
        ntile = math.ceil((B - l0) / TM_FWD)
        for pp in range(math.ceil(ntile / 4)):
            t0, nt = 4 * pp, min(4, ntile - 4 * pp)
            for c in range(nchunks):
                for tt in range(nt):
                    lb = l0 + TM_FWD * (t0 + tt)
                    rows = min(TM_FWD, B - lb)
                    for g in range(math.ceil(rows / G_FWD)):
                        yield (l0, c, lb, g, min(G_FWD, rows - g * G_FWD))


def fwd_converter(B, l0s):
    """(groups consumed, steps, data-operand cuts) in the converters' order."""
    n = 2 * B
    nchunks = math.ceil(n / KC_FWD)
    groups, steps, cuts = [], [], []
    for k, l0 in enumerate(l0s):
        ntile = math.ceil((B - l0) / TM_FWD)
        for pp in range(math.ceil(ntile / 4)):
            t0, nt = 4 * pp, min(4, ntile - 4 * pp)
            for c in range(nchunks):
                for tt in range(nt):
                    lb = l0 + TM_FWD * (t0 + tt)
                    rows = min(TM_FWD, B - lb)
                    if tt == 0:
                        cuts.append((k, l0, pp, c))
                    for g in range(math.ceil(rows / G_FWD)):
                        groups.append((l0, c, lb, g, min(G_FWD, rows - g * G_FWD)))
                    steps.append((k, l0, pp, c, tt, c == nchunks - 1))  # last flag: the tile's epilogue follows
    return groups, steps, cuts


def fwd_issuer(B, l0s):
    n = 2 * B
    nchunks = math.ceil(n / KC_FWD)
    out = []
    for l0 in l0s:
        ntile = math.ceil((B - l0) / TM_FWD)
        for pp in range(math.ceil(ntile / 4)):
            nt = min(4, ntile - 4 * pp)
            for c in range(nchunks):
                for tt in range(nt):
                    out.append((l0, pp, c, tt, 128 * tt, c == 0))
    return out


@pytest.mark.parametrize("B", [1, 2, 3, 8, 31, 64, 65, 100, 128, 200, 256, 300, 512])
def test_forward_roles_agree(B):
    grid = min(152, B * (B + 1) // 2)
    for cta in sorted({0, grid // 2, grid - 1}):
        l0s = clusters_of_cta(B, cta, grid)
        prod = list(fwd_producer(B, l0s))
        groups, steps, cuts = fwd_converter(B, l0s)
        iss = fwd_issuer(B, l0s)
        assert prod == groups
        assert len(steps) == len(iss)
        for (_, l0, pp, c, tt, _), (l0i, ppi, ci, tti, dcol, first) in zip(steps, iss):
            assert (l0, pp, c, tt) == (l0i, ppi, ci, tti)
            assert 0 <= dcol <= 3 * 128 and dcol + 112 <= 512  # the tile's accumulator in the 512 columns
            assert first == (c == 0)
        # every tile's accumulation closes exactly once (its epilogue), after its last chunk
        closes = [(k, pp, tt) for (k, l0, pp, c, tt, last) in steps if last]
        assert len(closes) == len(set(closes)) == sum(math.ceil((B - l0) / TM_FWD) for l0 in l0s)
        # the data operand is cut once per (cluster, pass, chunk), at the pass's first tile
        nchunks = math.ceil(2 * B / KC_FWD)
        assert len(cuts) == sum(math.ceil(math.ceil((B - l0) / TM_FWD) / 4) * nchunks for l0 in l0s)
        # a second pass only for clusters of more than 4 tiles (B = 512, L > 256)
        assert all(pp == 0 for (k, l0, pp, c) in cuts if B - l0 <= 4 * TM_FWD)


# ---- inverse -------------------------------------------------------------------
def inv_producer(B, l0s, tau):
    n = 2 * B
    npairs = math.ceil(n / (2 * TM_INV))
    for l0 in l0s:
        L = B - l0
        for jp in range(npairs):
            if 2 * TM_INV * jp + TM_INV * tau >= n:
                continue
            for c in range(math.ceil(L / KC_INV)):
                cnt = min(KC_INV, L - c * KC_INV)
                for g in range(math.ceil(cnt / 16)):
                    yield (l0, jp, c, g)


def inv_converter(B, l0s, tau):
    n = 2 * B
    npairs = math.ceil(n / (2 * TM_INV))
    groups, afull, waits = [], 0, 0
    pending = False
    for l0 in l0s:
        for jp in range(npairs):
            live = 2 * TM_INV * jp + TM_INV * tau < n
            lb, c = l0, 0
            while lb < B:
                cnt = min(KC_INV, B - lb)
                if pending:
                    waits += 1  # mdone[tau]
                if live:
                    for g in range(math.ceil(cnt / 16)):
                        groups.append((l0, jp, c, g))
                    afull += 1
                pending = live
                lb += KC_INV
                c += 1
    if pending:
        waits += 1
    return groups, afull, waits


def inv_issuer(B, l0s):
    n = 2 * B
    npairs = math.ceil(n / (2 * TM_INV))
    ready, per_tile = 0, [0, 0]
    for l0 in l0s:
        for jp in range(npairs):
            lb = l0
            while lb < B:
                ready += 1
                for tau in range(2):
                    if 2 * TM_INV * jp + TM_INV * tau >= n:
                        continue
                    per_tile[tau] += 1  # one afull wait and one mdone commit
                lb += KC_INV
    return ready, per_tile


@pytest.mark.parametrize("B", [1, 2, 5, 16, 63, 64, 65, 80, 96, 128, 160, 192, 256, 320, 512])
def test_inverse_roles_agree(B):
    grid = min(152, B * (B + 1) // 2)
    for cta in sorted({0, grid // 2, grid - 1}):
        l0s = clusters_of_cta(B, cta, grid)
        ready, per_tile = inv_issuer(B, l0s)
        steps = sum(math.ceil(2 * B / (2 * TM_INV)) * math.ceil((B - l0) / KC_INV) for l0 in l0s)
        assert ready == steps  # one ready per converter step
        for tau in range(2):
            prod = list(inv_producer(B, l0s, tau))
            groups, afull, waits = inv_converter(B, l0s, tau)
            assert prod == groups
            assert afull == per_tile[tau] == waits
            if 2 * B <= TM_INV:  # one sample tile: the second slot never runs
                assert (tau == 0) or (not prod and afull == 0)
