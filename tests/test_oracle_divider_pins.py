"""Pins of the oracle's per-row divider (both sides) and of its margin output
(no GPU).

The divider is defined by Def. 2.1 (a cell is red when its continuation value
is at least its exercise value) and located by Cor. 2.7 and the BSM boundary
theorem (Sec. 4.2): calls report the last red column of each row, puts the
last green one.  The margin is min |continuation - exercise| over the divider
cell and the cell right of it; parity tests use it to excuse ties.

Three independent pins:
  * the red/green colour of every node of the non-recombining tree (brute
    force over all paths, T <= 11 binomial, T <= 7 trinomial and BSM) gives
    each row's divider without any lattice code;
  * on the full grid (whose values brute force pins elsewhere), the
    continuation of every cell rebuilt here from the row above: the divider
    cell has the colour the definition asks, every cell right of it the other
    one, and the margin is the distance at the two cells next to the divider;
  * divider arrays shifted by one cell either way, and margins read at the
    wrong pair of cells, fail the grid check.
"""
import math

import numpy as np
import pytest

NONE_PUT = -(2 ** 31)
CALLS = (0, 1)
LATTICE_PUTS = (3, 4)


def _req(model, T, rng, tri_form=0, q_zero=False):
    lam = math.sqrt(3) if (model in (1, 4) and tri_form == 0) else 0.0
    q = 0.0 if (model == 2 or q_zero) else rng.uniform(0.005, 0.06)
    return dict(model=model, S0=rng.uniform(60, 140), K=rng.uniform(60, 140), r=rng.uniform(0.01, 0.08),
                q=q, sigma=rng.uniform(0.1, 0.6), expiry=rng.uniform(0.1, 3.0), T=T, lam=lam,
                tri_form=tri_form)


# ----------------------------------------------------------- brute force
def _tree_colours(level_max, steps, exercise, is_put):
    """Walk every path of the non-recombining tree from the root (level 0)
    and return {(level, x): list of (continuation - exercise)} over all nodes
    reaching that state.  Leaves have continuation 0."""
    seen = {}

    def value(level, x):
        ex = exercise(level, x)
        if level == level_max:
            cont = 0.0
        else:
            cont = 0.0
            for w, mv in steps:
                cont += w * value(level + 1, x + mv)
        seen.setdefault((level, x), []).append(cont - ex)
        return max(cont, ex) if level < level_max else max(ex, 0.0)

    value(0, 0)
    return seen


def _brute_dividers(req, P, tol):
    """Divider of every grid row from the tree's colours.  Returns (div,
    ambiguous) with ambiguous[row] True when a decisive node of that row is
    within tol of a tie (then the row is not compared)."""
    T, model = req["T"], req["model"]
    S, K = req["S0"], req["K"]
    if model == 2:
        s0 = math.log(S / K)
        b, c, a = P["w"]
        steps = [(a, +1), (c, 0), (b, -1)]
        ex = lambda lvl, k: 1.0 - math.exp(s0 + k * P["ds"])
    else:
        m, u = P["m"], P["u"]
        if P["D"] == 1:
            steps = [(m * P["p"], +1), (m * (1 - P["p"]), -1)]
        else:
            steps = [(m * P["pu"], +1), (m * P["po"], 0), (m * P["pd"], -1)]
        sign = -1.0 if model in LATTICE_PUTS else 1.0
        ex = lambda lvl, x: sign * (S * math.exp(x * P["logu"]) - K)
    put = model == 2 or model in LATTICE_PUTS
    seen = _tree_colours(T, steps, ex, put)
    div = {}
    amb = {}
    for (level, x), diffs in seen.items():
        # grid row and column of the node
        if model == 2:
            row, col = T - level, x            # BSM: row n = T - level, index k
        elif P["D"] == 1:
            row, col = level, (x + level) // 2
        else:
            row, col = level, x + level
        d = np.asarray(diffs)
        if put:
            mark = d < 0                        # green: exercise > continuation
        else:
            mark = d >= 0                       # red: continuation >= exercise
        if np.any(np.abs(d) <= tol):
            amb[row] = True
        if mark.all() != mark.any():            # paths disagree: a tie within rounding
            amb[row] = True
        if mark.all():
            div[row] = max(div.get(row, -(10 ** 9)), col)
    none = NONE_PUT if model == 2 else -1
    out = np.full(T + 1, none, dtype=np.int64)
    for row, col in div.items():
        out[row] = col
    ambiguous = np.zeros(T + 1, dtype=bool)
    for row in amb:
        ambiguous[row] = True
    return out, ambiguous


CASES_BRUTE = [(0, 0, T) for T in (2, 5, 8, 11)] + [(3, 0, T) for T in (2, 5, 8, 11)] + \
    [(1, f, T) for f in (0, 1) for T in (3, 5, 7)] + [(4, f, T) for f in (0, 1) for T in (3, 7)] + \
    [(2, 0, T) for T in (3, 5, 7)]


@pytest.mark.parametrize("model,form,T", CASES_BRUTE)
def test_divider_matches_nonrecombining_tree(oracle_lib, model, form, T):
    """Each row's divider equals the last red (call) or last green (put) node
    of that row on the non-recombining tree, for several random options."""
    rng = np.random.default_rng(4000 + 97 * model + 13 * form + T)
    compared = 0
    for _ in range(4):
        req = _req(model, T, rng, tri_form=form)
        P = oracle_lib.params(req)
        _, bnd, _ = oracle_lib.price_american(req, with_boundary=True, with_margin=True)
        scale = 1.0 if model == 2 else req["K"]
        want, amb = _brute_dividers(req, P, 1e-12 * scale)
        for row in range(T + 1):
            if amb[row]:
                continue
            assert bnd[row] == want[row], (req, row, bnd[row], want[row])
            compared += 1
    assert compared >= 2 * (T + 1)


# ------------------------------------------------------------ grid checks
def _continuation(g, req, P):
    """Continuation value of every cell, rebuilt from the row above in the
    oracle's grid (row T of a lattice, row 0 of the BSM grid: 0)."""
    T = req["T"]
    cont = np.full_like(g, np.nan)
    if req["model"] == 2:
        b, c, a = P["w"]
        cont[0, :] = 0.0
        for n in range(1, T + 1):
            R = T - n
            k = np.arange(-R, R + 1) + T
            prev = g[n - 1]
            cont[n, k] = b * prev[k - 1] + c * prev[k] + a * prev[k + 1]
    else:
        D = P["D"]
        w = P["w"]
        cont[T, :] = 0.0
        for i in range(T):
            j = np.arange(D * i + 1)
            nxt = g[i + 1]
            v = w[0] * nxt[j] + w[1] * nxt[j + 1]
            if D == 2:
                v = v + w[2] * nxt[j + 2]
            cont[i, j] = v
    return cont


def _exercise(req, P):
    T, S, K = req["T"], req["S0"], req["K"]
    if req["model"] == 2:
        k = np.arange(-T, T + 1)
        return np.broadcast_to(1.0 - np.exp(math.log(S / K) + k * P["ds"]), (T + 1, 2 * T + 1))
    D = P["D"]
    ex = np.full((T + 1, D * T + 1), np.nan)
    sign = -1.0 if req["model"] in LATTICE_PUTS else 1.0
    for i in range(T + 1):
        j = np.arange(D * i + 1)
        x = (2 * j - i) if D == 1 else (j - i)
        ex[i, j] = sign * (S * np.exp(x * P["logu"]) - K)
    return ex


def divider_violations(req, P, g, bnd, margin, tol):
    """Rows whose divider or margin contradicts the definition on the grid.
    A decision closer than tol to a tie is not held against the divider."""
    T, model = req["T"], req["model"]
    cont = _continuation(g, req, P)
    ex = _exercise(req, P)
    put = model == 2 or model in LATTICE_PUTS
    bad = []
    for row in range(T + 1):
        if model == 2:
            R = T - row
            cols = np.arange(-R, R + 1)
            idx = cols + T
            none = NONE_PUT
        else:
            cols = np.arange(P["D"] * row + 1)
            idx = cols
            none = -1
        d = cont[row, idx] - ex[row, idx]           # >= 0: red, < 0: green
        mark = (d < 0) if put else (d >= 0)         # the colour the divider reports
        sure = np.abs(d) > tol
        b = bnd[row]
        pos = -1 if b == none else int(b - cols[0])  # position of the divider in cols
        if pos >= len(cols) or pos < -1:
            bad.append((row, "divider outside the row"))
            continue
        if pos >= 0 and sure[pos] and not mark[pos]:
            bad.append((row, "divider cell has the wrong colour"))
        right = slice(pos + 1, len(cols))
        if np.any(mark[right] & sure[right]):
            bad.append((row, "a cell right of the divider has the divider's colour"))
        # margin: |cont - ex| at the divider cell and the next one (those in the row)
        pair = [p for p in (pos, pos + 1) if 0 <= p < len(cols)]
        want = min(abs(d[p]) for p in pair) if pair else math.inf
        got = margin[row]
        if not (got == want or abs(got - want) <= 1e-9 * max(abs(want), 1e-300) + 1e-14 * tol / 1e-12):
            bad.append((row, "margin %r, want %r" % (got, want)))
    return bad


CASES_GRID = [(0, 0), (1, 0), (1, 1), (3, 0), (4, 0), (4, 1), (2, 0)]


def _grid_case(oracle_lib, model, form, seed, T=None):
    rng = np.random.default_rng(4200 + 31 * model + 7 * form + seed)
    req = _req(model, T or int(rng.integers(30, 140)), rng, tri_form=form)
    P = oracle_lib.params(req)
    g, gb = oracle_lib.grid(req)
    _, bnd, margin = oracle_lib.price_american(req, with_boundary=True, with_margin=True)
    assert np.array_equal(gb, bnd)
    tol = 1e-12 * (1.0 if model == 2 else req["K"])
    return req, P, g, bnd, margin, tol


@pytest.mark.parametrize("model,form", CASES_GRID)
@pytest.mark.parametrize("seed", range(3))
def test_divider_and_margin_on_grid(oracle_lib, model, form, seed):
    """The divider cell has the reported colour, every cell right of it the
    other one, and the margin is the distance to a tie at the divider cell and
    the cell right of it -- for every row of the grid."""
    req, P, g, bnd, margin, tol = _grid_case(oracle_lib, model, form, seed)
    assert divider_violations(req, P, g, bnd, margin, tol) == []


@pytest.mark.parametrize("model,form", CASES_GRID)
def test_grid_check_rejects_planted_mistakes(oracle_lib, model, form):
    """A divider one cell too far right or left, or a margin read at the cell
    pair left of the right one, fails the grid check on some row."""
    req, P, g, bnd, margin, tol = _grid_case(oracle_lib, model, form, 0, T=120)
    none = NONE_PUT if model == 2 else -1
    live = bnd != none
    for shift in (+1, -1):
        moved = bnd.copy()
        moved[live] += shift
        assert divider_violations(req, P, g, moved, margin, tol), shift
    # margin read at (divider - 1, divider) instead of (divider, divider + 1)
    cont = _continuation(g, req, P)
    ex = _exercise(req, P)
    wrong = margin.copy()
    for row in range(req["T"] + 1):
        b = bnd[row]
        if b == none:
            continue
        col0 = -(req["T"] - row) if model == 2 else 0
        off = req["T"] if model == 2 else 0
        cells = [c for c in (b - 1, b) if c >= col0]
        if cells:
            wrong[row] = min(abs(cont[row, c + off] - ex[row, c + off]) for c in cells)
    assert divider_violations(req, P, g, bnd, wrong, tol)
