"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test ties the oracle to something other than itself: brute force on the
non-recombining tree, closed-form European sums, the Black-Scholes limit, the
American-call-without-dividends identity, the paper's weight identities and
its structural lemmas on the red/green divider.  The puts on the binomial and
trinomial lattices and the BSM put with a dividend yield (variants the paper
does not treat) are pinned the same way, plus the exact put-call symmetry of
the lattice (an American put equals the American call with spot and strike
and rate and yield exchanged; McDonald and Schroder, 1998).
"""
import math

import numpy as np
import pytest

from tests import closed_forms as cf
from paper_2303_02317_gb300 import workloads as wl

RNG = np.random.default_rng(7)


def _rand_req(model, T, rng, q_zero=False, tri_form=0, bsm_yield=False):
    S0 = rng.uniform(50, 150)
    K = rng.uniform(50, 150)
    sigma = rng.uniform(0.1, 0.6)
    r = rng.uniform(0.0, 0.08)
    q = 0.0 if (q_zero or (model == 2 and not bsm_yield)) else rng.uniform(0.005, 0.06)
    E = rng.uniform(0.1, 3.0)
    lam = math.sqrt(3) if (model in (1, 4) and tri_form == 0) else 0.0
    return dict(model=model, S0=S0, K=K, r=r, q=q, sigma=sigma, expiry=E, T=T, lam=lam,
                tri_form=tri_form)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(6))
def test_bopm_matches_nonrecombining_tree(oracle_lib, seed):
    """Fig. 1 lattice == every path of the binomial tree (Sec. 2.1)."""
    rng = np.random.default_rng(100 + seed)
    for T in (1, 2, 5, 11):
        req = _rand_req(0, T, rng)
        P = oracle_lib.params(req)
        u, p, m = P["u"], P["p"], P["m"]
        steps = [(m * p, +1), (m * (1 - p), -1)]
        ex = lambda lvl, x: req["S0"] * u ** x - req["K"]
        bf = cf.brute_force_tree(T, steps, ex, 0)
        got = oracle_lib.price_american(req)
        assert got == pytest.approx(bf, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("tri_form", [0, 1])
def test_topm_matches_nonrecombining_tree(oracle_lib, tri_form):
    """Trinomial lattice (Sec. 3) == every path of the trinomial tree."""
    rng = np.random.default_rng(200 + tri_form)
    for T in (1, 3, 7):
        req = _rand_req(1, T, rng, tri_form=tri_form)
        P = oracle_lib.params(req)
        u, m = P["u"], P["m"]
        steps = [(m * P["pu"], +1), (m * P["po"], 0), (m * P["pd"], -1)]
        ex = lambda lvl, x: req["S0"] * u ** x - req["K"]
        bf = cf.brute_force_tree(T, steps, ex, 0)
        assert oracle_lib.price_american(req) == pytest.approx(bf, rel=1e-13, abs=1e-13)


def test_bsm_matches_nonrecombining_walk(oracle_lib):
    """The explicit scheme (Sec. 4, bsmG) is a trinomial walk with weights
    (b, c, a) on (k-1, k, k+1); enumerate every path."""
    rng = np.random.default_rng(300)
    for T in (1, 4, 7):
        req = _rand_req(2, T, rng)
        P = oracle_lib.params(req)
        b, c, a = P["w"]
        ds = P["ds"]
        steps = [(a, +1), (c, 0), (b, -1)]
        s0 = math.log(req["S0"] / req["K"])
        ex = lambda lvl, k: 1.0 - math.exp(s0 + k * ds)
        bf = req["K"] * cf.brute_force_tree(T, steps, ex, 0)
        assert oracle_lib.price_american(req) == pytest.approx(bf, rel=1e-13, abs=1e-13)


# -------------------------------------------------------------- closed forms
def test_weight_identities(oracle_lib):
    """Sec. 2 (proof of Lemma 2.2): s0/u + s1 u = e^{-Y dt}; the same
    martingale identity m (p_d/u + p_o + p_u u) = e^{-Y dt} for both
    trinomial forms; BSM: c = 1 - a - b - omega dtau with a + b = 2/3."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        req = _rand_req(0, int(rng.integers(10, 5000)), rng)
        P = oracle_lib.params(req)
        sd, su = P["w"]
        assert sd / P["u"] + su * P["u"] == pytest.approx(math.exp(-req["q"] * P["dt"]), rel=1e-14)
        for form in (0, 1):
            t = _rand_req(1, int(rng.integers(10, 5000)), rng, tri_form=form)
            Q = oracle_lib.params(t)
            wd, wo, wu = Q["w"]
            lhs = wd / Q["u"] + wo + wu * Q["u"]
            assert lhs == pytest.approx(math.exp(-t["q"] * Q["dt"]), rel=1e-13)
            if form == 0:   # Boyle: second moment matched too
                m2 = (wd / Q["u"] ** 2 + wo + wu * Q["u"] ** 2) / Q["m"]
                assert m2 == pytest.approx(math.exp((2 * (t["r"] - t["q"]) + t["sigma"] ** 2) * Q["dt"]), rel=1e-12)
            else:           # paper form: two binomial half steps, p_u = p^2, p_d = (1-p)^2
                p = math.sqrt(Q["pu"])
                assert Q["pd"] == pytest.approx((1 - p) ** 2, rel=1e-12)
        s = _rand_req(2, int(rng.integers(10, 5000)), rng)
        B = oracle_lib.params(s)
        b, c, a = B["w"]
        assert a + b == pytest.approx(2.0 / 3.0, rel=1e-14)
        assert c == pytest.approx(1.0 / 3.0 - B["omega"] * B["dtau"], rel=1e-12)


@pytest.mark.parametrize("T", [16, 301, 2048])
def test_binomial_call_without_yield_is_european_sum(oracle_lib, T):
    """With Y=0 Lemma 2.3's bound is infinite: no interior green cell, so the
    American call equals the European binomial sum."""
    rng = np.random.default_rng(T)
    for _ in range(3):
        req = _rand_req(0, T, rng, q_zero=True)
        P = oracle_lib.params(req)
        ref = cf.binomial_european_call(req["S0"], req["K"], T, P["u"], P["p"], P["m"])
        assert oracle_lib.price_american(req) == pytest.approx(ref, rel=1e-11, abs=1e-12)
        assert oracle_lib.price_european(req) == pytest.approx(ref, rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("tri_form", [0, 1])
def test_trinomial_call_without_yield_is_european_sum(oracle_lib, tri_form):
    rng = np.random.default_rng(41 + tri_form)
    for T in (9, 120):
        req = _rand_req(1, T, rng, q_zero=True, tri_form=tri_form)
        P = oracle_lib.params(req)
        ref = cf.trinomial_european_call(req["S0"], req["K"], T, P["u"], P["pu"], P["po"], P["pd"], P["m"])
        assert oracle_lib.price_american(req) == pytest.approx(ref, rel=1e-11, abs=1e-12)


def test_european_lattices_converge_to_black_scholes(oracle_lib):
    """European values on the three lattices approach the Black-Scholes
    closed form as T grows (error O(1/T))."""
    rng = np.random.default_rng(5)
    for _ in range(3):
        req = _rand_req(0, 4096, rng)
        ref = cf.bs_call(req["S0"], req["K"], req["r"], req["q"], req["sigma"], req["expiry"])
        assert abs(oracle_lib.price_european(req) - ref) < 2e-3 * req["K"] / 100 + 1e-3
        for form in (0, 1):
            t = dict(req, model=1, tri_form=form, lam=math.sqrt(3) if form == 0 else 0.0)
            assert abs(oracle_lib.price_european(t) - ref) < 2e-3 * req["K"] / 100 + 1e-3
        p = dict(req, model=2, q=0.0)
        refp = cf.bs_put(p["S0"], p["K"], p["r"], 0.0, p["sigma"], p["expiry"])
        assert abs(oracle_lib.price_european(p) - refp) < 2e-3 * req["K"] / 100 + 1e-3


def test_bsm_put_without_rate_has_no_early_exercise(oracle_lib):
    """r = 0 (omega = 0): the explicit scheme keeps the continuation above
    the payoff, so American == European, and both approach Black-Scholes."""
    rng = np.random.default_rng(9)
    for T in (64, 1000):
        req = _rand_req(2, T, rng)
        req["r"] = 0.0
        am = oracle_lib.price_american(req)
        eu = oracle_lib.price_european(req)
        assert am == pytest.approx(eu, rel=1e-13, abs=1e-14)
    req = _rand_req(2, 4096, rng)
    req["r"] = 0.0
    ref = cf.bs_put(req["S0"], req["K"], 0.0, 0.0, req["sigma"], req["expiry"])
    assert abs(oracle_lib.price_american(req) - ref) < 2e-3


def test_american_bounds(oracle_lib):
    """max(European on the same lattice, intrinsic) <= American;
    call <= S0; put <= K (the price lies between the European price and
    these no-arbitrage caps)."""
    for req in wl.random_small(30, seed=3, T_range=(5, 400)):
        d = req.as_dict()
        am = oracle_lib.price_american(d)
        eu = oracle_lib.price_european(d)
        if req.model == 2:
            intr = max(req.K - req.S0, 0.0)
            assert am <= req.K + 1e-12
        else:
            intr = max(req.S0 - req.K, 0.0)
            assert am <= req.S0 + 1e-12
        assert am >= eu - 1e-12 * max(1.0, eu)
        assert am >= intr - 1e-12 * max(1.0, intr)


# ----------------------------------------------------------- divider lemmas
def _call_checks(oracle_lib, req):
    g, bnd = oracle_lib.grid(req)
    P = oracle_lib.params(req)
    T, D = req["T"], P["D"]
    S, K = req["S0"], req["K"]
    u = P["u"]
    for i in range(T - 1):
        # Cor. 2.7 / its trinomial analogue: the divider moves <= 1 cell left,
        # except that a fully red row is clipped at the row end (D i).
        assert min(bnd[i + 1] - 1, D * i) <= bnd[i] <= bnd[i + 1], (i, bnd[i], bnd[i + 1])
    for i in range(T + 1):
        row = g[i, : D * i + 1]
        # hidden lemma of Sec. 2.2 (trinomial: row monotone): non-decreasing rows
        assert np.all(np.diff(row) >= -1e-12 * max(1.0, np.max(np.abs(row))))
        # red cells left of the divider, green (== exercise) right of it
        k = np.arange(D * i + 1)
        ex = S * np.exp(P["logu"] * ((2 * k - i) if D == 1 else (k - i))) - K
        green = k > bnd[i]
        assert np.allclose(row[green], np.maximum(ex[green], 0.0 if i == T else ex[green]), rtol=1e-13, atol=1e-13)
    if D == 1:
        # Lemma timedecay: G[i][j] >= G[i+2][j+1]
        for i in range(T - 1):
            for j in range(i):
                assert g[i, j] >= g[i + 2, j + 1] - 1e-12
        # Lemma 2.3: a green cell of row i < T sits at or right of the bound
        if req["q"] > 0 and req["r"] > 0:
            dt = P["dt"]
            shift = math.log((K / S) * (1 - math.exp(-req["r"] * dt)) / (1 - math.exp(-req["q"] * dt)))
            for i in range(T):
                if bnd[i] < i:
                    assert bnd[i] + 1 >= i / 2 + shift / (2 * req["sigma"] * math.sqrt(dt)) - 1e-9
    else:
        # trinomial diagonal lemma: G[i+1][j+1] <= G[i][j]
        for i in range(T - 1):
            for j in range(2 * i + 1):
                assert g[i + 1, j + 1] <= g[i, j] + 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_call_divider_lemmas(oracle_lib, seed):
    rng = np.random.default_rng(500 + seed)
    for model, form in ((0, 0), (1, 0), (1, 1)):
        req = _rand_req(model, int(rng.integers(20, 160)), rng, tri_form=form)
        _call_checks(oracle_lib, req)


@pytest.mark.parametrize("seed", range(4))
def test_bsm_divider_theorem(oracle_lib, seed):
    """BSM boundary theorem: 0 <= k_n - k_{n+1} <= 1, green left of the
    divider holds the payoff, red right of it holds the continuation."""
    rng = np.random.default_rng(600 + seed)
    req = _rand_req(2, int(rng.integers(20, 200)), rng)
    g, bnd = oracle_lib.grid(req)
    T = req["T"]
    P = oracle_lib.params(req)
    s0 = math.log(req["S0"] / req["K"])
    NONE = oracle_lib.INT32_MIN
    for n in range(1, T):      # from row 1: see test_bsm_expiry_row_exception
        if bnd[n] == NONE:
            continue
        if bnd[n + 1] != NONE:
            assert 0 <= bnd[n] - bnd[n + 1] <= 1, (n, bnd[n], bnd[n + 1])
        else:
            # the divider left the shrinking triangle on its left edge
            assert bnd[n] - 1 < -(T - n - 1)
    for n in range(T + 1):
        R = T - n
        k = np.arange(-R, R + 1)
        row = g[n, k + T]
        ex = 1 - np.exp(s0 + k * P["ds"])
        green = k <= (bnd[n] if bnd[n] != NONE else -R - 1)
        assert np.allclose(row[green], ex[green], rtol=1e-13, atol=1e-13)
        assert np.all(row >= np.maximum(ex, 0.0) - 1e-13)


def test_invalid_inputs_rejected(oracle_lib):
    base = wl.fixed_call(0, 64).as_dict()
    for bad in (dict(S0=0.0), dict(K=-1.0), dict(sigma=0.0), dict(expiry=0.0), dict(T=0),
                dict(model=5), dict(model=-1)):
        assert oracle_lib.status_of(dict(base, **bad)) == 1
    assert oracle_lib.status_of(dict(wl.fixed_bsm_put(64).as_dict(), q=0.01)) == 0
    # r - q so large at tiny sigma that p > 1
    assert oracle_lib.status_of(dict(base, sigma=0.001, r=0.5, T=4)) == 2


def test_bsm_expiry_row_exception(oracle_lib):
    """The divider theorem's proof uses a divider cell that is green through
    the max at row n; at the expiry row (n = 0) cells are green by their payoff
    alone, so the step 0 -> 1 can move the divider by many cells (r = 0: no
    cell stays green at all, the American put equals the European one).  From
    row 1 on the theorem holds again."""
    r0 = dict(model=2, S0=100.0, K=100.0, r=0.0, q=0.0, sigma=0.3, expiry=1.0, T=400)
    _, b, _ = oracle_lib.price_american(r0, with_boundary=True, with_margin=True)
    assert b[0] == -1 and (b[1:] == oracle_lib.INT32_MIN).all()
    r1 = dict(r0, r=1e-6, sigma=0.6, expiry=3.0)
    _, b, _ = oracle_lib.price_american(r1, with_boundary=True, with_margin=True)
    assert b[0] - b[1] > 1
    live = [(b[n], b[n + 1]) for n in range(1, 400) if b[n + 1] != oracle_lib.INT32_MIN]
    assert live and all(0 <= x - y <= 1 for x, y in live)


# ------------------------------------------- puts on the lattices, BSM yield
@pytest.mark.parametrize("seed", range(3))
def test_lattice_puts_match_nonrecombining_tree(oracle_lib, seed):
    """Binomial and trinomial puts (exercise value K - S u^x) == every path."""
    rng = np.random.default_rng(700 + seed)
    for T in (1, 2, 5, 11):
        req = _rand_req(3, T, rng)
        P = oracle_lib.params(req)
        u, p, m = P["u"], P["p"], P["m"]
        ex = lambda lvl, x: req["K"] - req["S0"] * u ** x
        bf = cf.brute_force_tree(T, [(m * p, +1), (m * (1 - p), -1)], ex, 0)
        assert oracle_lib.price_american(req) == pytest.approx(bf, rel=1e-13, abs=1e-13)
    for form in (0, 1):
        for T in (1, 3, 7):
            req = _rand_req(4, T, rng, tri_form=form)
            P = oracle_lib.params(req)
            u, m = P["u"], P["m"]
            ex = lambda lvl, x: req["K"] - req["S0"] * u ** x
            steps = [(m * P["pu"], +1), (m * P["po"], 0), (m * P["pd"], -1)]
            bf = cf.brute_force_tree(T, steps, ex, 0)
            assert oracle_lib.price_american(req) == pytest.approx(bf, rel=1e-13, abs=1e-13)


def test_bsm_with_yield_matches_nonrecombining_walk(oracle_lib):
    """With a yield the scheme keeps the walk form (weights b, c, a) with
    a - b = (omega_y - 1) dtau/ds, omega_y = 2(r - q)/sigma^2, a + b = 2/3 and
    c = 1 - a - b - omega dtau; enumerate every path."""
    rng = np.random.default_rng(310)
    for T in (1, 4, 7):
        req = _rand_req(2, T, rng, bsm_yield=True)
        P = oracle_lib.params(req)
        b, c, a = P["w"]
        dtau, ds = P["dtau"], P["ds"]
        om = 2 * req["r"] / req["sigma"] ** 2
        omy = 2 * (req["r"] - req["q"]) / req["sigma"] ** 2
        assert a - b == pytest.approx((omy - 1) * dtau / ds, rel=1e-12, abs=1e-15)
        assert a + b == pytest.approx(2.0 / 3.0, rel=1e-14)
        assert c == pytest.approx(1.0 / 3.0 - om * dtau, rel=1e-12)
        s0 = math.log(req["S0"] / req["K"])
        ex = lambda lvl, k: 1.0 - math.exp(s0 + k * ds)
        bf = req["K"] * cf.brute_force_tree(T, [(a, +1), (c, 0), (b, -1)], ex, 0)
        assert oracle_lib.price_american(req) == pytest.approx(bf, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("T", [12, 257, 2048])
def test_put_call_symmetry_on_the_lattice(oracle_lib, T):
    """On the binomial lattice (u d = 1) and on the paper's trinomial form (two
    binomial half steps) the American put with (S, K, r, q) equals the American
    call with (K, S, q, r) exactly (McDonald and Schroder, 1998): dividing the
    put by the node price turns its recursion into the call's.  The Boyle form
    matches two moments only, so there the identity holds to O(dt) alone."""
    rng = np.random.default_rng(800 + T)
    for model, form in ((0, 0), (1, 1)):
        for _ in range(3):
            put = _rand_req(model + 3, T, rng, tri_form=form)
            call = dict(put, model=model, S0=put["K"], K=put["S0"], r=put["q"], q=put["r"])
            assert oracle_lib.price_american(put) == pytest.approx(
                oracle_lib.price_american(call), rel=5e-12, abs=1e-12)
            assert oracle_lib.price_european(put) == pytest.approx(
                oracle_lib.price_european(call), rel=5e-12, abs=1e-12)


@pytest.mark.parametrize("T", [16, 301])
def test_lattice_puts_without_rate_are_european_sums(oracle_lib, T):
    """r = 0: exercising a put early earns no interest on the strike, so the
    American put equals the European lattice sum (binomial and trinomial)."""
    rng = np.random.default_rng(900 + T)
    for _ in range(2):
        req = dict(_rand_req(3, T, rng), r=0.0)
        P = oracle_lib.params(req)
        ref = cf.binomial_european_put(req["S0"], req["K"], T, P["u"], P["p"], P["m"])
        assert oracle_lib.price_american(req) == pytest.approx(ref, rel=1e-11, abs=1e-12)
    for form in (0, 1):
        req = dict(_rand_req(4, min(T, 120), rng, tri_form=form), r=0.0)
        P = oracle_lib.params(req)
        ref = cf.trinomial_european_put(req["S0"], req["K"], req["T"], P["u"], P["pu"], P["po"], P["pd"], P["m"])
        assert oracle_lib.price_american(req) == pytest.approx(ref, rel=1e-11, abs=1e-12)


def test_european_put_call_parity_and_black_scholes_limit(oracle_lib):
    """European lattice values obey C - P = S e^{-q E} - K e^{-r E} exactly
    (the lattices match the first moment), and the European puts (lattices and
    BSM with a yield) approach the Black-Scholes put as T grows."""
    rng = np.random.default_rng(13)
    for model, form in ((0, 0), (1, 0), (1, 1)):
        req = _rand_req(model, 777, rng, tri_form=form)
        put = dict(req, model=model + 3)
        fwd = req["S0"] * math.exp(-req["q"] * req["expiry"]) - req["K"] * math.exp(-req["r"] * req["expiry"])
        diff = oracle_lib.price_european(req) - oracle_lib.price_european(put)
        assert diff == pytest.approx(fwd, rel=1e-11, abs=1e-11 * req["K"])
    for model, form in ((3, 0), (4, 0), (4, 1), (2, 0)):
        req = _rand_req(model, 4096, rng, tri_form=form, bsm_yield=True)
        ref = cf.bs_put(req["S0"], req["K"], req["r"], req["q"], req["sigma"], req["expiry"])
        assert abs(oracle_lib.price_european(req) - ref) < 2e-3 * req["K"] / 100 + 1e-3


def test_bsm_put_with_yield_and_no_rate_has_no_early_exercise(oracle_lib):
    rng = np.random.default_rng(19)
    for T in (64, 1000):
        req = dict(_rand_req(2, T, rng, bsm_yield=True), r=0.0)
        assert oracle_lib.price_american(req) == pytest.approx(oracle_lib.price_european(req),
                                                               rel=1e-13, abs=1e-14)


def test_put_bounds(oracle_lib):
    """max(European, intrinsic) <= American put <= K for every put model."""
    reqs = wl.random_small(30, seed=23, T_range=(5, 400), models=(3, 4, 2), bsm_yield=True)
    for req in reqs:
        d = req.as_dict()
        am = oracle_lib.price_american(d)
        eu = oracle_lib.price_european(d)
        intr = max(req.K - req.S0, 0.0)
        assert am <= req.K + 1e-12
        assert am >= eu - 1e-12 * max(1.0, eu)
        assert am >= intr - 1e-12 * max(1.0, intr)


@pytest.mark.parametrize("seed", range(4))
def test_lattice_put_divider(oracle_lib, seed):
    """Mirror image of Cor. 2.7: the green (exercise) cells of a put row are
    the columns 0..b_i, and the divider steps by D or D-1 columns per row
    toward the root (b_i in [b_{i+1} - D, b_{i+1} - D + 1], clipped at -1);
    put rows are non-increasing in j."""
    rng = np.random.default_rng(1000 + seed)
    for model, form in ((3, 0), (4, 0), (4, 1)):
        req = _rand_req(model, int(rng.integers(20, 160)), rng, tri_form=form)
        g, bnd = oracle_lib.grid(req)
        P = oracle_lib.params(req)
        T, D = req["T"], P["D"]
        for i in range(T - 1):
            lo, hi = bnd[i + 1] - D, bnd[i + 1] - D + 1
            assert lo <= bnd[i] <= hi or (bnd[i] == -1 and hi <= 0), (i, bnd[i], bnd[i + 1])
        for i in range(T + 1):
            row = g[i, : D * i + 1]
            assert np.all(np.diff(row) <= 1e-12 * max(1.0, np.max(np.abs(row))))
            k = np.arange(D * i + 1)
            ex = req["K"] - req["S0"] * np.exp(P["logu"] * ((2 * k - i) if D == 1 else (k - i)))
            green = k <= bnd[i]
            assert np.allclose(row[green], ex[green], rtol=1e-13, atol=1e-13)
            assert np.all(row[~green] >= ex[~green] - 1e-12 * req["K"])


@pytest.mark.parametrize("seed", range(4))
def test_bsm_divider_theorem_with_yield(oracle_lib, seed):
    """The BSM boundary theorem (0 <= k_n - k_{n+1} <= 1 from row 1 on, green
    left of the divider) checked on the yield variant the paper does not prove."""
    rng = np.random.default_rng(1100 + seed)
    req = _rand_req(2, int(rng.integers(20, 200)), rng, bsm_yield=True)
    g, bnd = oracle_lib.grid(req)
    T = req["T"]
    P = oracle_lib.params(req)
    s0 = math.log(req["S0"] / req["K"])
    NONE = oracle_lib.INT32_MIN
    for n in range(1, T):
        if bnd[n] != NONE and bnd[n + 1] != NONE:
            assert 0 <= bnd[n] - bnd[n + 1] <= 1, (n, bnd[n], bnd[n + 1])
    for n in range(T + 1):
        R = T - n
        k = np.arange(-R, R + 1)
        row = g[n, k + T]
        ex = 1 - np.exp(s0 + k * P["ds"])
        green = k <= (bnd[n] if bnd[n] != NONE else -R - 1)
        assert np.allclose(row[green], ex[green], rtol=1e-13, atol=1e-13)
        assert np.all(row >= np.maximum(ex, 0.0) - 1e-13)


# ----------------------------------------------------------- sensitivities
def test_greek_rows_match_nonrecombining_tree(oracle_lib):
    """The nodes next to the root that the sensitivities read equal the
    brute-force value of the sub-tree rooted at each of them."""
    rng = np.random.default_rng(1200)
    for model, form in ((0, 0), (3, 0), (1, 0), (4, 1)):
        T = 7 if model in (0, 3) else 5
        req = _rand_req(model, T, rng, tri_form=form)
        P = oracle_lib.params(req)
        u, m = P["u"], P["m"]
        put = model in (3, 4)
        ex = (lambda lvl, x: req["K"] - req["S0"] * u ** x) if put else (lambda lvl, x: req["S0"] * u ** x - req["K"])
        if P["D"] == 1:
            steps = [(m * P["p"], +1), (m * (1 - P["p"]), -1)]
            nodes = [(1, 2 * j - 1, j) for j in range(2)] + [(2, 2 * j - 2, 3 + j) for j in range(3)]
        else:
            steps = [(m * P["pu"], +1), (m * P["po"], 0), (m * P["pd"], -1)]
            nodes = [(1, j - 1, j) for j in range(3)] + [(2, j - 2, 3 + j) for j in range(5)]
        (price, _, _, _), near = oracle_lib.greeks(req)
        assert price == pytest.approx(oracle_lib.price_american(req), rel=1e-15)
        for lvl, x, slot in nodes:
            bf = cf.brute_force_tree(T - lvl, steps, ex, x)
            assert near[slot] == pytest.approx(bf, rel=1e-13, abs=1e-13), (model, lvl, x)
    req = _rand_req(2, 6, rng, bsm_yield=True)
    P = oracle_lib.params(req)
    b, c, a = P["w"]
    s0 = math.log(req["S0"] / req["K"])
    ex = lambda lvl, k: 1.0 - math.exp(s0 + k * P["ds"])
    _, near = oracle_lib.greeks(req)
    for back, ks, base in ((1, range(-1, 2), 0), (2, range(-2, 3), 3)):
        for i, k in enumerate(ks):
            bf = cf.brute_force_tree(req["T"] - back, [(a, +1), (c, 0), (b, -1)], ex, k)
            assert near[base + i] == pytest.approx(bf, rel=1e-13, abs=1e-13)


def test_greeks_of_european_lattice_are_differences_of_closed_forms(oracle_lib):
    """q = 0 binomial call (no early exercise): each node next to the root is
    the European binomial sum of the sub-lattice below it (T-1 or T-2 steps
    from spot S u^x), so the sensitivities are differences of closed forms."""
    rng = np.random.default_rng(1300)
    for T in (9, 300):
        req = _rand_req(0, T, rng, q_zero=True)
        P = oracle_lib.params(req)
        u, p, m, S, K = P["u"], P["p"], P["m"], req["S0"], req["K"]
        E = lambda s, n: cf.binomial_european_call(s, K, n, u, p, m)
        (price, delta, gamma, theta), _ = oracle_lib.greeks(req)
        g10, g11 = E(S / u, T - 1), E(S * u, T - 1)
        g20, g21, g22 = E(S / u ** 2, T - 2), E(S, T - 2), E(S * u ** 2, T - 2)
        assert delta == pytest.approx((g11 - g10) / (S * u - S / u), rel=1e-9)
        up, dn = (g22 - g21) / (S * u ** 2 - S), (g21 - g20) / (S - S / u ** 2)
        assert gamma == pytest.approx((up - dn) / ((S * u ** 2 - S / u ** 2) / 2), rel=1e-7)
        assert theta == pytest.approx((g21 - E(S, T)) / (2 * P["dt"]), rel=1e-8)


def test_greeks_black_scholes_limit(oracle_lib):
    """Without early exercise (q = 0 calls, r = 0 puts) the lattice
    sensitivities approach the Black-Scholes-Merton ones as T grows."""
    rng = np.random.default_rng(1400)
    for model, form in ((0, 0), (1, 0), (1, 1), (3, 0), (4, 0), (4, 1), (2, 0)):
        call = model in (0, 1)
        req = _rand_req(model, 4096, rng, tri_form=form, q_zero=call, bsm_yield=True)
        req["S0"], req["K"] = rng.uniform(75, 125), 100.0
        if not call:
            req["r"] = 0.0
        (_, d, g, t), _ = oracle_lib.greeks(req)
        bd, bg, bt = cf.bs_greeks(req["S0"], req["K"], req["r"], req["q"], req["sigma"], req["expiry"], call)
        assert abs(d - bd) < 1e-3, (model, d, bd)
        assert abs(g - bg) < 2e-3 * bg, (model, g, bg)
        assert abs(t - bt) < 2e-3 * abs(bt) + 1e-4, (model, t, bt)


def test_american_greeks_satisfy_the_pde_at_the_root(oracle_lib):
    """Where the root lies in the continuation region the American value
    solves the Black-Scholes-Merton equation there:
    theta + sigma^2 S^2 gamma / 2 + (r - q) S delta - r V = 0 (to O(dt))."""
    rng = np.random.default_rng(1500)
    for model, form in ((3, 0), (4, 0), (4, 1), (2, 0), (0, 0), (1, 1)):
        req = _rand_req(model, 4096, rng, tri_form=form, bsm_yield=True)
        req["r"], req["q"] = rng.uniform(0.02, 0.08), rng.uniform(0.005, 0.05)
        req["K"] = 100.0
        req["S0"] = rng.uniform(95, 125) if model in (2, 3, 4) else rng.uniform(75, 105)
        (v, d, g, t), _ = oracle_lib.greeks(req)
        S = req["S0"]
        res = t + 0.5 * req["sigma"] ** 2 * S * S * g + (req["r"] - req["q"]) * S * d - req["r"] * v
        assert abs(res) < 3e-3 * req["r"] * v, (model, res, v)


# ------------------------------------------------ the linear advance (Sec. 2.3)

def _unit_response(oracle, w, h, W):
    """Row of the h-step advance's kernel: the advance of unit rows e_j."""
    eye = np.eye(W)
    return oracle.linear_advance(eye, w, h)[:, 0]      # output cell 0 sees input j with weight k_j


def test_linear_advance_binomial_coefficients(oracle_lib):
    """Two-point stencil: output cell y sees input y + j with weight
    C(h, j) w0^(h-j) w1^j (the binomial distribution of h up-moves)."""
    from math import comb
    w, h = (0.37, 0.61), 23
    k = _unit_response(oracle_lib, w, h, h + 1)
    want = np.array([comb(h, j) * w[0] ** (h - j) * w[1] ** j for j in range(h + 1)])
    assert np.allclose(k, want, rtol=1e-13, atol=0.0)


def test_linear_advance_trinomial_coefficients(oracle_lib):
    """Three-point stencil: the weight of offset j is the multinomial sum
    over a + b + c = h, b + 2c = j of h!/(a! b! c!) w0^a w1^b w2^c."""
    from math import factorial
    w, h = (0.21, 0.5, 0.28), 9
    k = _unit_response(oracle_lib, w, h, 2 * h + 1)
    want = np.zeros(2 * h + 1)
    for c in range(h + 1):
        for b in range(h - c + 1):
            a = h - b - c
            want[b + 2 * c] += factorial(h) // (factorial(a) * factorial(b) * factorial(c)) * \
                w[0] ** a * w[1] ** b * w[2] ** c
    assert np.allclose(k, want, rtol=1e-13, atol=0.0)


def test_linear_advance_constant_row_and_shape(oracle_lib):
    """A constant row stays constant times (sum w)^h; W cells give
    W - (len(w) - 1) h cells."""
    for w, h in (((0.4, 0.55), 17), ((0.2, 0.3, 0.45), 11)):
        x = np.full((2, 200), 3.5)
        y = oracle_lib.linear_advance(x, w, h)
        assert y.shape == (2, 200 - (len(w) - 1) * h)
        assert np.allclose(y, 3.5 * sum(w) ** h, rtol=1e-14, atol=0.0)
