"""GPU GA generation against the oracle: bit-exact operators given the same
fitness vector and Philox key, the stateful pipeline's wiring generation by
generation, initial populations, termination, and end-to-end recovery."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import assert_L_close, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1403_4099_gb300 import build, gpga
    build.build()
    return gpga


def _gparams(g, P, E=2, **kw):
    return g.default_params(P=P, elite=E, **kw)


def _oparams(orc, gp, N):
    return orc.params(gp.P, N, elite=gp.elite, max_gens=gp.max_gens, stall_gens=gp.stall_gens,
                      tol=gp.tol, pc=gp.pc, pkb=gp.pkb, pm=gp.pm, scaling=gp.scaling,
                      init_labels=gp.init_labels)


CASES = [
    # P, N, E, pc, pkb, pm, scaling, generation
    (64, 16, 2, 0.9, 0.9, 0.01, 0, 0),
    (1000, 100, 10, 0.9, 0.9, 0.1, 0, 7),
    (37, 5, 0, 1.0, 0.5, 0.2, 0, 3),
    (4096, 500, 10, 0.9, 0.9, 0.01, 0, 12345),
    (333, 65, 5, 0.7, 0.3, 0.05, 1, 2),
    (2, 2, 1, 1.0, 1.0, 1.0, 0, 1),
    (129, 31, 128, 0.9, 0.9, 0.5, 1, 9),
    (16384, 40, 10, 0.9, 0.9, 0.05, 0, 5),  # the largest population accepted
]


@pytest.mark.parametrize("case", CASES)
def test_evolve_bit_exact(g, orc, case):
    import torch
    P, N, E, pc, pkb, pm, scaling, gen = case
    rng = np.random.default_rng(P + N)
    pop = rng.integers(0, N, (P, N)).astype(np.int32)
    L = np.round(rng.standard_normal(P) * 3, 2)  # ties
    L[rng.integers(0, P, 3)] = -np.inf
    L[rng.integers(0, P)] = np.nan
    if scaling == 1:
        L = np.abs(np.nan_to_num(L, nan=0.5, neginf=0.0))
    seed = 0xDEADBEEF12345 + P
    gp = _gparams(g, P, E, pc=pc, pkb=pkb, pm=pm, scaling=scaling)
    nxt, perm, par = g.ga_evolve(dev(pop, torch.int32), dev(L), gp, seed, gen)
    torch.cuda.synchronize()
    onxt, operm, opar = orc.ga_evolve(pop, L, _oparams(orc, gp, N), seed, gen)
    assert np.array_equal(perm.cpu().numpy(), operm)
    if P - E:
        assert np.array_equal(par.cpu().numpy(), opar)
    assert np.array_equal(nxt.cpu().numpy(), onxt)


@pytest.mark.parametrize("P", [2, 33, 1000, 4096, 16384])
@pytest.mark.parametrize("dist", ["equal", "narrow", "outliers", "signed_zero_nan"])
def test_rank_order_adversarial_fitness(g, orc, P, dist):
    """The device's rank order (key descending, index ascending, NaN as -inf)
    equals the oracle's for fitness vectors that crowd the keys together or
    spread them apart: all equal, a spread of 1e-9 around 75, a few huge
    outliers, and signed zeros with NaN and infinities, from the smallest
    population to the largest accepted."""
    import torch
    rng = np.random.default_rng(P * 7 + len(dist))
    if dist == "equal":
        L = np.full(P, 3.25)
    elif dist == "narrow":
        L = 75.0 + rng.random(P) * 1e-9
        L[rng.integers(0, P, P // 4 + 1)] = 75.0
    elif dist == "outliers":
        L = rng.standard_normal(P)
        L[rng.integers(0, P, 2)] = 1e300
        L[rng.integers(0, P, 2)] = -1e300
    else:
        L = np.round(rng.standard_normal(P), 1)
        L[rng.integers(0, P, P // 8 + 1)] = 0.0
        L[rng.integers(0, P, P // 8 + 1)] = -0.0
        L[rng.integers(0, P, 3)] = np.nan
        L[rng.integers(0, P, 2)] = -np.inf
        L[rng.integers(0, P, 2)] = np.inf
    N = 8
    pop = rng.integers(0, N, (P, N)).astype(np.int32)
    E = min(2, P - 1)
    gp = _gparams(g, P, E)
    _, perm, _ = g.ga_evolve(dev(pop, torch.int32), dev(L), gp, 99, 4)
    torch.cuda.synchronize()
    assert np.array_equal(perm.cpu().numpy(), orc.ga_rank(L))


def test_uniform_init_bit_exact(g, orc):
    import torch
    p = synth.n100()
    C = orc.pearson(p.R)
    for K0 in (0, 13):
        gp = _gparams(g, 300, init_labels=K0)
        ga = g.GA(dev(C), gp, seed=99)
        pop, L = ga.population()
        assert np.array_equal(pop, orc.ga_init(300, 100, 99, K0=K0 or None))
        assert_L_close(L, orc.loglik_batch(pop, C), "gen0")
        ga.close()


def test_threshold_init_bit_exact(g, orc):
    for which in ("n100", "small16", "n500"):
        p = getattr(synth, which)()
        C = orc.pearson(p.R)
        gp = _gparams(g, 257, init=g.INIT_THRESHOLD, tau_lo=0.05, tau_hi=0.6)
        ga = g.GA(dev(C), gp, seed=1234)
        pop, _ = ga.population()
        assert np.array_equal(pop, orc.ga_init_threshold(C, 257, 1234, 0.05, 0.6))
        ga.close()


@pytest.mark.parametrize("scaling,form", [(0, 0), (1, 0), (0, 2), (1, 2), (0, 1)])
def test_pipeline_generation_by_generation(g, orc, scaling, form):
    """Each device generation equals the oracle's operators applied to the
    device's own population and fitness (bit-exact), and the device fitness
    matches the oracle's likelihood of that population."""
    p = synth.n100()
    C = orc.pearson(p.R)
    gp = _gparams(g, 1024, E=10, scaling=scaling, max_gens=50, tol=-1.0, record=1, form=form)
    seed = 4242
    ga = g.GA(dev(C), gp, seed=seed)
    op = _oparams(orc, gp, 100)
    pop, L = ga.population()
    for gen in range(8):
        assert_L_close(L, orc.loglik_batch(pop, C), f"gen {gen}")
        ref_next, _, _ = orc.ga_evolve(pop, L, op, seed, gen)
        ga.step(1)
        pop, L = ga.population()
        assert np.array_equal(pop, ref_next), f"generation {gen + 1}"
    h = ga.history()
    assert len(h["best_L"]) == 9 and np.all(np.diff(h["best_L"]) >= 0)
    assert np.all(np.diff(h["t_ns"]) >= 0)
    lab, Lb, gen = ga.best()
    assert gen == 8
    assert np.array_equal(lab, orc.canonicalize(lab))
    assert abs(Lb - orc.loglik(lab, C)) <= 1e-10 * max(1, abs(Lb))
    assert abs(Lb - h["best_L"][-1]) <= 1e-4 + 1e-6 * abs(Lb)
    ga.close()


def test_termination_and_noop_after_done(g, orc):
    p = synth.small16()
    C = orc.pearson(p.R)
    gp = _gparams(g, 64, max_gens=5, tol=-1.0)
    ga = g.GA(dev(C), gp, seed=5)
    assert ga.step(3, wait=True) is False
    assert ga.step(2, wait=True) is True
    pop5, L5 = ga.population()
    ga.step(4, wait=True)
    pop9, L9 = ga.population()
    assert np.array_equal(pop5, pop9) and np.array_equal(L5, L9)
    assert ga.best()[2] == 5
    ga.close()
    # stall rule: a huge tolerance stops at generation G_stall
    gp = _gparams(g, 64, max_gens=100, stall_gens=4, tol=1e9)
    ga = g.GA(dev(C), gp, seed=5)
    assert ga.step(10, wait=True) is True
    assert ga.best()[2] == 4
    ga.close()


@pytest.mark.parametrize("form", [0, 1, 2])
def test_recovers_small16(g, orc, form):
    p = synth.small16()
    C = orc.pearson(p.R)
    gp = _gparams(g, 64, max_gens=200, tol=-1.0, form=form)
    ga = g.GA(dev(C), gp, seed=synth.seed_for(1))
    ga.step(200)
    lab, L, gen = ga.best()
    assert gen == 200
    assert orc.ari(lab, p.truth) >= 0.99
    ga.close()


@pytest.mark.parametrize("form", [0, 2])
def test_global_max_n10(g, orc, form):
    """Small-workload parameters on N=10: the exhaustive maximum in >= 99 of
    100 seeds."""
    p = synth.small10()
    C = orc.pearson(p.R)
    _, Lmax, _ = orc.brute_force(C)
    gp = _gparams(g, 64, max_gens=200, tol=-1.0, form=form)
    ga = g.GA(dev(C), gp, seed=1)
    hits = 0
    for k in range(100):
        ga.reset(dev(C), 1000 + k)
        ga.step(200)
        _, L, _ = ga.best()
        hits += abs(L - Lmax) <= 1e-9 * abs(Lmax)
    ga.close()
    assert hits >= 99


def test_bad_params_rejected(g, orc):
    C = orc.pearson(synth.small16().R)
    for kw in (dict(P=1), dict(elite=64), dict(pm=1.5), dict(scaling=7), dict(form=9)):
        gp = _gparams(g, 64)
        for k, v in kw.items():
            setattr(gp, k, v)
        with pytest.raises(g.GpgaError) as e:
            g.GA(dev(C), gp, seed=1)
        assert e.value.code == g.ERR_ARG


@pytest.fixture(scope="module")
def n500_C(orc):
    p = synth.n500()
    return p, orc.pearson(p.R)


@pytest.mark.parametrize("init", ["uniform", "threshold"])
def test_headline_path_generation_by_generation_n500(g, orc, n500_C, init):
    """The path the benchmark times, at its own size: gather form, 16-bit
    labels, the fused generation kernel with the SUS bracket table of the rank
    prefix, N=500, P=4096, E=10, P_m=0.01/gene. Each device generation equals
    the oracle's operators applied to the device's own population and fitness
    (bit-exact), and every device L is within 1e-4 + 1e-6|L| of the oracle's
    Eq. 8. The threshold start has clusters of well over 8 members, so the
    warp-wide big-cluster pair sums are exercised as well as the per-lane ones.
    Then the 8-generation graph the benchmark launches is checked against 8
    single-generation launches of a twin run."""
    p, C = n500_C
    kw = dict(init=g.INIT_THRESHOLD, tau_lo=0.05, tau_hi=0.6) if init == "threshold" else {}
    gp = _gparams(g, 4096, E=10, max_gens=60, tol=-1.0, pm=0.01, form=g.FORM_GATHER, **kw)
    seed = 14034099
    ga = g.GA(dev(C), gp, seed=seed)
    op = _oparams(orc, gp, 500)
    pop, L = ga.population()
    biggest = 0
    for gen in range(5):
        assert_L_close(L, orc.loglik_batch(pop, C), f"{init} gen {gen}")
        biggest = max(biggest, max(np.bincount(row).max() for row in pop[:64]))
        ref_next, _, _ = orc.ga_evolve(pop, L, op, seed, gen)
        ga.step(1)
        pop, L = ga.population()
        assert np.array_equal(pop, ref_next), f"{init}: generation {gen + 1}"
    assert_L_close(L, orc.loglik_batch(pop, C), f"{init} gen 5")
    if init == "threshold":
        assert biggest > 8
    # the 8-generation graph against single generations, from the same start
    twin = g.GA(dev(C), gp, seed=seed)
    ga.step(8)
    for _ in range(5 + 8):
        twin.step(1)
    pa, La = ga.population()
    pb, Lb = twin.population()
    assert np.array_equal(pa, pb) and np.array_equal(La, Lb)
    assert_L_close(La, orc.loglik_batch(pa, C), f"{init} gen 13")
    ga.close()
    twin.close()


def test_delta_scores_equal_full_scores(g, orc):
    """From DELTA_MIN_N (448) genes up a run scores most children by delta
    from a parent's score table; ga_score scores the same configurations from
    scratch in the same per-cluster form. After several generations (the
    tables carried from generation to generation) every fitness value of the
    population must equal ga_score's bit for bit, from a uniform and from a
    clustered start."""
    import torch
    pl = synth.market_clusters(2, 460, 1840, 38, 0.2, 0.8, replicate=11)
    C = orc.pearson(pl.R)
    for init in (g.INIT_UNIFORM, g.INIT_THRESHOLD):
        gp = _gparams(g, 512, E=10, max_gens=40, tol=-1.0, pm=0.01, form=g.FORM_GATHER, init=init)
        ga = g.GA(dev(C), gp, seed=909)
        for steps in (1, 7, 12):
            ga.step(steps)
            pop, L = ga.population()
            full = g.ga_score(dev(pop, torch.int32), dev(C), form=g.FORM_GATHER)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(L, full.cpu().numpy())
            assert_L_close(L, orc.loglik_batch(pop, C), f"delta L vs oracle, init {init}")
        ga.close()
