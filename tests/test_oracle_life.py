"""Pins for the oracle's Game of Life loop (Fig. 1 elemental function, B3/S23).

The pins are catalogue facts of Conway's Life (tests/golden/life_patterns.txt,
with its citation), the torus wrap (a glider crosses an N x N torus and is back
after 4N generations), a dead-border case worked out by hand, and the loop
semantics of Sec. 3.1 (repeat-until on the "any cell changed" reduce, live
count reduce, cap).
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "life_patterns.txt")


def load_patterns():
    pats, cur = {}, None
    for line in open(GOLDEN):
        line = line.rstrip("\n")
        if not line or line.startswith("#"):
            continue
        if line.startswith("pattern "):
            parts = line.split()
            cur = {"name": parts[1], "kind": parts[2], "n": int(parts[3]),
                   "shift": tuple(int(x) for x in parts[4:6]) if len(parts) > 4 else None,
                   "rows": []}
            pats[cur["name"]] = cur
        else:
            cur["rows"].append([1 if ch == "O" else 0 for ch in line])
    for p in pats.values():
        p["cells"] = np.array(p["rows"], dtype=np.uint8)
    return pats


PATTERNS = load_patterns()


def place(pattern, n=32, at=(12, 12)):
    g = np.zeros((n, n), dtype=np.uint8)
    ph, pw = pattern.shape
    g[at[0]:at[0] + ph, at[1]:at[1] + pw] = pattern
    return g


@pytest.mark.parametrize("name", [k for k, v in PATTERNS.items() if v["kind"] == "still"])
def test_still_lifes_stop_after_one_generation(orc, name):
    g = place(PATTERNS[name]["cells"])
    out, r = orc.life(g, wrap=True, max_gens=100)
    assert r.iters == 1 and r.converged and not r.changed
    assert np.array_equal(out, g)
    assert r.count == int(g.sum())


@pytest.mark.parametrize("name", [k for k, v in PATTERNS.items() if v["kind"] == "osc"])
def test_oscillators_have_their_period(orc, name):
    pat = PATTERNS[name]
    g = place(pat["cells"])
    for k in range(1, pat["n"]):
        out, r = orc.life(g, wrap=True, max_gens=k)
        assert not np.array_equal(out, g) and r.changed and not r.converged
    out, r = orc.life(g, wrap=True, max_gens=pat["n"])
    assert np.array_equal(out, g) and r.iters == pat["n"] and not r.converged


def test_glider_moves_one_cell_diagonally_every_four_generations(orc):
    pat = PATTERNS["glider"]
    g = place(pat["cells"], n=24, at=(5, 5))
    out, r = orc.life(g, wrap=True, max_gens=pat["n"])
    assert np.array_equal(out, np.roll(g, pat["shift"], axis=(0, 1)))
    assert r.count == 5


@pytest.mark.parametrize("n", [8, 13])
def test_glider_crosses_torus_and_returns(orc, n):
    g = place(PATTERNS["glider"]["cells"], n=n, at=(2, 3))
    out, _ = orc.life(g, wrap=True, max_gens=4 * n)
    assert np.array_equal(out, g)
    half, _ = orc.life(g, wrap=True, max_gens=2 * n)
    assert not np.array_equal(half, g)


def test_diehard_vanishes_after_130_generations(orc):
    g = place(PATTERNS["diehard"]["cells"], n=96, at=(44, 44))
    out, r = orc.life(g, wrap=True, max_gens=129)
    assert out.sum() > 0
    out, r = orc.life(g, wrap=True, max_gens=130)
    assert out.sum() == 0 and r.count == 0
    # one more generation leaves the empty grid unchanged: the loop stops there
    out, r = orc.life(g, wrap=True, max_gens=1000)
    assert r.iters == 131 and r.converged


def test_dead_border_blinker_worked_by_hand(orc):
    # Horizontal blinker on the top row of an 8 x 8 grid with a dead border
    # (Fig. 1 boundary): generation 1 keeps the centre (2 neighbours) and births
    # the cell below it (3 neighbours); generation 2 is empty (each of the two
    # cells has 1 neighbour, no cell has 3); generation 3 changes nothing.
    g = np.zeros((8, 8), dtype=np.uint8)
    g[0, 3:6] = 1
    g1, r1 = orc.life(g, wrap=False, max_gens=1)
    expect = np.zeros_like(g)
    expect[0, 4] = expect[1, 4] = 1
    assert np.array_equal(g1, expect) and r1.count == 2
    g3, r3 = orc.life(g, wrap=False, max_gens=50)
    assert r3.iters == 3 and r3.converged and r3.count == 0 and g3.sum() == 0
    # on the torus the same cells form an ordinary period-2 blinker
    gw, rw = orc.life(g, wrap=True, max_gens=2)
    assert np.array_equal(gw, g) and rw.changed


def test_lone_cell_and_crowded_cell_die(orc):
    g = np.zeros((7, 7), dtype=np.uint8)
    g[3, 3] = 1
    out, _ = orc.life(g, wrap=True, max_gens=1)
    assert out.sum() == 0
    # a plus sign: the centre has 4 neighbours and dies; the four tips have 3
    # live neighbours at the diagonal gaps, so those 4 cells are born
    g = np.zeros((7, 7), dtype=np.uint8)
    g[3, 2:5] = 1
    g[2:5, 3] = 1
    out, _ = orc.life(g, wrap=True, max_gens=1)
    assert out[3, 3] == 0
    assert all(out[y, x] == 1 for y, x in ((2, 2), (2, 4), (4, 2), (4, 4)))


def test_random_soup_count_and_cap(orc):
    from paper_1609_04567_gb300 import inputs
    g = inputs.life_cells(40, 56, seed=1)
    out, r = orc.life(g, wrap=True, max_gens=25)
    assert r.count == int(out.sum())
    assert r.iters <= 25
    # resuming equals running straight through (the loop is deterministic)
    mid, _ = orc.life(g, wrap=True, max_gens=10)
    out2, _ = orc.life(mid, wrap=True, max_gens=15)
    assert np.array_equal(out, out2)


def test_life_is_equivariant_under_torus_symmetries(orc):
    from paper_1609_04567_gb300 import inputs
    g = inputs.life_cells(24, 24, seed=2)
    out, _ = orc.life(g, wrap=True, max_gens=12)
    sh, _ = orc.life(np.roll(g, (5, -7), axis=(0, 1)), wrap=True, max_gens=12)
    assert np.array_equal(sh, np.roll(out, (5, -7), axis=(0, 1)))
    tr, _ = orc.life(g.T, wrap=True, max_gens=12)
    assert np.array_equal(tr, out.T)


def _next_by_definition(g, wrap):
    """Conway's rule applied from its statement, independently of the oracle:
    a dead cell with exactly three live neighbours is born, a live cell with two
    or three survives, every other cell is dead next.  Neighbours are the eight
    cells at offsets (dy, dx) != (0, 0), |dy|, |dx| <= 1, taken modulo the
    extents on the torus and dead outside the grid otherwise."""
    ny, nx = g.shape
    out = np.zeros_like(g)
    for y in range(ny):
        for x in range(nx):
            n = 0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dy == 0 and dx == 0:
                        continue
                    yy, xx = y + dy, x + dx
                    if wrap:
                        n += int(g[yy % ny, xx % nx] != 0)
                    elif 0 <= yy < ny and 0 <= xx < nx:
                        n += int(g[yy, xx] != 0)
            alive = g[y, x] != 0
            out[y, x] = 1 if (n in (2, 3) if alive else n == 3) else 0
    return out


def test_rule_table_over_all_512_neighbourhoods(orc):
    # Each of the 2^9 states of a 3 x 3 block (bit 4 = the centre) placed side
    # by side: a block's centre sees only its own block, so one generation of
    # the whole grid evaluates the rule on every neighbourhood at once.
    rows, cols = 16, 32
    g = np.zeros((3 * rows, 3 * cols), dtype=np.uint8)
    for cfg in range(512):
        by, bx = divmod(cfg, cols)
        for b in range(9):
            g[3 * by + b // 3, 3 * bx + b % 3] = (cfg >> b) & 1
    for wrap in (True, False):
        out, _ = orc.life(g, wrap=wrap, max_gens=1)
        for cfg in range(512):
            by, bx = divmod(cfg, cols)
            alive = (cfg >> 4) & 1
            n = bin(cfg & ~(1 << 4)).count("1")
            born_or_survives = n == 3 or (alive == 1 and n == 2)
            assert out[3 * by + 1, 3 * bx + 1] == int(born_or_survives), (cfg, wrap)


@pytest.mark.parametrize("shape,wrap", [((8, 8), True), ((8, 8), False), ((7, 13), True), ((5, 9), False)])
def test_brute_force_generations_on_small_grids(orc, shape, wrap):
    # Generation by generation against the rule evaluated from its statement,
    # with the loop's reduces: the live count and whether any cell changed.
    from paper_1609_04567_gb300 import inputs
    g = inputs.life_cells(shape[0], shape[1], seed=5 + shape[1])
    for _ in range(12):
        expect = _next_by_definition(g, wrap)
        out, r = orc.life(g, wrap=wrap, max_gens=1)
        assert np.array_equal(out, expect)
        assert r.iters == 1 and r.count == int(expect.sum())
        assert bool(r.changed) == bool((expect != g).any())
        assert bool(r.converged) == (not (expect != g).any())
        g = out
