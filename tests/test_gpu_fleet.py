"""Batched runs and the serving loop: every run of a fleet must give exactly
(bit for bit) the result of the same run alone through ga_init / ga_step /
ga_best, whatever other runs share the device, the launch shape the tuner
picked, the order of admission or the memory budget."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth

pytestmark = pytest.mark.gpu


def _params(gpga, P=128, max_gens=40, stall=10, tol=1e-5, **kw):
    return gpga.default_params(P=P, elite=4, max_gens=max_gens, stall_gens=stall, tol=tol,
                               pm=0.01, form=gpga.FORM_GATHER, **kw)


def _single(gpga, C, prm, seed):
    ga = gpga.GA(C, prm, seed=seed)
    ga.step(prm.max_gens)
    lab, L, g = ga.best()
    ga.close()
    return lab, L, g


def _corr(gpga, R):
    import torch
    Rt = torch.from_numpy(np.ascontiguousarray(R)).cuda()
    return gpga.cluster_corr(Rt)


@pytest.fixture(scope="module")
def gpga():
    from paper_1403_4099_gb300 import gpga as g
    g.lib()
    return g


def _windows(gpga, Ns, rep=0):
    Cs = []
    for k, n in enumerate(Ns):
        pl = synth.market_clusters(2, n, 4 * n, max(2, n // 12), 0.2, 0.8, replicate=100 + rep + k)
        Cs.append(_corr(gpga, pl.R))
    return Cs


def test_batch_matches_single_runs(gpga):
    Ns = [17, 40, 64, 65, 100, 129, 23]
    Cs = _windows(gpga, Ns)
    seeds = [11 + 7 * k for k in range(len(Ns))]
    prm = _params(gpga)
    b = gpga.Batch(Cs, prm, seeds)
    tune = b.tuning()
    assert tune["warps_per_cta"] in (2, 4, 8, 16) and tune["ctas"] > 0 and tune["ms"] > 0
    active = b.step(3)
    assert 0 <= active <= len(Ns)
    while b.step(8) > 0:
        pass
    gens, done, best = b.status()
    assert done.all()
    for k, C in enumerate(Cs):
        lab, L, g = _single(gpga, C, prm, seeds[k])
        lb, Lb, gb = b.best(k)
        assert gb == g == gens[k], (k, gb, g, gens[k])
        np.testing.assert_array_equal(lb, lab)
        assert Lb == L, (k, Lb, L)
    b.close()


def test_batch_long_runs_match_single_runs(gpga):
    """Seventy generations without the stall rule, runs with clusters large
    enough for the warp-wide pair sums: every run still equals the same run
    alone, bit for bit, down to its whole final population and fitness."""
    Ns = [100, 160, 48]
    Cs = _windows(gpga, Ns, rep=7)
    seeds = [5 + 3 * k for k in range(len(Ns))]
    prm = _params(gpga, P=256, max_gens=70, tol=-1.0)
    b = gpga.Batch(Cs, prm, seeds)
    while b.step(8) > 0:
        pass
    gens, done, _ = b.status()
    assert done.all() and (gens == 70).all()
    for k, C in enumerate(Cs):
        ga = gpga.GA(C, prm, seed=seeds[k])
        ga.step(prm.max_gens)
        lab, L, g = ga.best()
        pop, Lpop = ga.population()
        ga.close()
        lb, Lb, gb = b.best(k)
        assert gb == g == 70
        np.testing.assert_array_equal(lb, lab)
        assert Lb == L, (k, Lb, L)
        pop_b, Lpop_b = b.population(k)
        np.testing.assert_array_equal(pop_b, pop)
        np.testing.assert_array_equal(Lpop_b, Lpop)
    b.close()


def test_batch_column_subsets(gpga):
    import torch
    win = synth.intraday(N=120, windows=4, W=390, stride=30)
    R = win.R[:390]
    Cfull = _corr(gpga, R)
    subs = synth.window_subsets(120, 3, nmin=20, nmax=120)
    cols = [torch.from_numpy(s).cuda() for s in subs]
    prm = _params(gpga, max_gens=24, tol=-1.0)
    seeds = [5, 6, 7]
    b = gpga.Batch([Cfull] * 3, prm, seeds, cols=cols)
    b.step(24)
    for k, s in enumerate(subs):
        Csub = Cfull[torch.from_numpy(s).long().cuda()][:, torch.from_numpy(s).long().cuda()]
        lab, L, g = _single(gpga, Csub.contiguous(), prm, seeds[k])
        lb, Lb, gb = b.best(k)
        assert gb == g == 24
        np.testing.assert_array_equal(lb, lab)
        assert Lb == L
    b.close()


def test_batch_rejects_other_forms(gpga):
    Cs = _windows(gpga, [20])
    prm = _params(gpga)
    prm.form = gpga.FORM_PLAIN
    with pytest.raises(gpga.GpgaError):
        gpga.Batch(Cs, prm, [1])


def _serve_all(gpga, srv, reqs, per_tick=1, gens=8):
    """Submit `per_tick` requests per tick (arrivals while others run) and
    collect every result."""
    ids = []
    pending = list(reqs)
    out = {}
    for _ in range(10000):
        for _ in range(per_tick):
            if pending:
                C, seed = pending.pop(0)
                ids.append(srv.submit(C, seed))
        srv.tick(gens)
        for i in ids:
            if i not in out:
                r = srv.result(i)
                if r is not None:
                    out[i] = r
        if not pending and len(out) == len(ids):
            break
    return [out[i] for i in ids]


def test_serving_alone_equals_mix(gpga):
    Ns = [30, 100, 30, 64, 100, 45]
    Cs = _windows(gpga, Ns, rep=40)
    Ch = [C.cpu().numpy() for C in Cs]
    prm = _params(gpga, P=256, max_gens=48, stall=12)
    seeds = [100 + k for k in range(len(Ns))]
    alone = []
    for C, s in zip(Ch, seeds):
        srv = gpga.Server(prm, max_runs=1, max_n=128)
        alone.append(_serve_all(gpga, srv, [(C, s)])[0])
        srv.close()
    # the mix: three slots, arrivals while others run, queueing
    srv = gpga.Server(prm, max_runs=3, max_n=128)
    mix = _serve_all(gpga, srv, list(zip(Ch, seeds)), per_tick=2, gens=8)
    st = srv.stats()
    assert st["completed"] == len(Ns) and st["bytes_in_use"] == 0
    srv.close()
    for k in range(len(Ns)):
        la, La, ga, _ = alone[k]
        lm, Lm, gm, (qs, rs) = mix[k]
        np.testing.assert_array_equal(lm, la)
        assert Lm == La and gm == ga
        assert qs >= 0 and rs >= 0
        lab, L, g = _single(gpga, Cs[k], prm, seeds[k])
        np.testing.assert_array_equal(la, lab)
        assert La == L and ga == g


def test_serving_admission_by_memory(gpga):
    Ns = [100, 100, 100]
    Cs = _windows(gpga, Ns, rep=60)
    Ch = [C.cpu().numpy() for C in Cs]
    prm = _params(gpga, P=256, max_gens=16, tol=-1.0)
    # a budget that holds one run of N=100 at a time: the others wait in the queue
    probe = gpga.Server(prm, max_runs=4, max_n=128)
    probe.submit(Ch[0], 1)
    probe.tick(0)
    one = probe.stats()["bytes_in_use"]
    probe.close()
    assert one > 0
    srv = gpga.Server(prm, max_runs=4, max_n=128, mem_budget=int(one * 1.5))
    for k, C in enumerate(Ch):
        srv.submit(C, 7 + k)
    active, queued = srv.tick(4)
    assert active == 1 and queued == 2
    assert srv.stats()["bytes_in_use"] <= int(one * 1.5)
    res = {}
    for _ in range(1000):
        srv.tick(4)
        for i in range(3):
            if i not in res:
                r = srv.result(i)
                if r is not None:
                    res[i] = r
        if len(res) == 3:
            break
    assert len(res) == 3
    for k in range(3):
        lab, L, g = _single(gpga, Cs[k], prm, 7 + k)
        np.testing.assert_array_equal(res[k][0], lab)
        assert res[k][1] == L and res[k][2] == g == 16
    with pytest.raises(gpga.GpgaError):
        srv.result(0)  # already collected
    srv.close()


@pytest.mark.parametrize("Ns", [[160, 23], [23, 160, 64]])
def test_batch_generation_by_generation_against_oracle(gpga, orc, Ns):
    """Each run of a fleet, generation by generation, against the oracle
    directly (not only against the same run alone): the next population is
    the oracle's operators applied to the run's own population and fitness
    (bit-exact), and every L is within 1e-4 + 1e-6|L| of the oracle's Eq. 8."""
    from gpu_util import assert_L_close
    Cs = _windows(gpga, Ns, rep=90)
    Ch = [C.cpu().numpy() for C in Cs]
    seeds = [31 + 5 * k for k in range(len(Ns))]
    prm = _params(gpga, P=192, max_gens=30, tol=-1.0)
    b = gpga.Batch(Cs, prm, seeds)
    ops = [orc.params(prm.P, n, elite=prm.elite, max_gens=prm.max_gens,
                      stall_gens=prm.stall_gens, tol=prm.tol, pc=prm.pc, pkb=prm.pkb, pm=prm.pm,
                      scaling=prm.scaling) for n in Ns]
    cur = [b.population(k) for k in range(len(Ns))]
    for gen in range(6):
        refs = []
        for k in range(len(Ns)):
            pop, L = cur[k]
            assert_L_close(L, orc.loglik_batch(pop, Ch[k]), f"run {k} gen {gen}")
            refs.append(orc.ga_evolve(pop, L, ops[k], seeds[k], gen)[0])
        b.step(1)
        cur = [b.population(k) for k in range(len(Ns))]
        for k in range(len(Ns)):
            assert np.array_equal(cur[k][0], refs[k]), f"run {k} (N={Ns[k]}) generation {gen + 1}"
    b.close()
