"""Island model: every device generation of every island equals the oracle's
operators applied to that island's device population and fitness, followed,
every migrate_every generations, by the oracle's ring migration (bit-exact
labels); migrants carry their fitness; with migration off the islands are
independent runs."""
import numpy as np
import pytest

from paper_1403_4099_gb300 import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1403_4099_gb300 import gpga
    gpga.lib()
    return gpga


def _params(g, orc, N, **kw):
    gp = g.default_params(P=128, elite=4, max_gens=400, tol=-1.0, pm=0.05,
                          form=g.FORM_GATHER, **kw)
    op = orc.params(gp.P, N, elite=gp.elite, max_gens=gp.max_gens, stall_gens=gp.stall_gens,
                    tol=gp.tol, pc=gp.pc, pkb=gp.pkb, pm=gp.pm, scaling=gp.scaling,
                    init_labels=gp.init_labels)
    return gp, op


@pytest.mark.parametrize("every,m", [(2, 2), (3, 4)])
def test_islands_generation_by_generation(g, orc, every, m):
    p = synth.n100(replicate=1)
    C = orc.pearson(p.R)
    gp, op = _params(g, orc, 100)
    K, seed = 3, 777
    b = g.Batch.islands(dev(C), gp, K, seed, every, m)
    pops = [b.population(k) for k in range(K)]
    for gen in range(7):
        nxt = np.stack([orc.ga_evolve(pops[k][0], pops[k][1], op, seed + k, gen)[0]
                        for k in range(K)])
        if (gen + 1) % every == 0:
            nxt, _ = orc.island_migrate(nxt, np.zeros((K, gp.P)), m)
        b.step(1)
        pops = [b.population(k) for k in range(K)]
        for k in range(K):
            assert np.array_equal(pops[k][0], nxt[k]), (gen + 1, k)
        if (gen + 1) % every == 0:  # migrants keep their fitness
            for k in range(K):
                np.testing.assert_array_equal(pops[(k + 1) % K][1][gp.P - m:], pops[k][1][:m])
    b.close()


def test_islands_without_migration_are_independent_runs(g, orc):
    p = synth.small16()
    C = orc.pearson(p.R)
    gp, _ = _params(g, orc, 16, )
    gp.max_gens = 30
    # migrate_every beyond max_gens: no migration ever happens
    b = g.Batch.islands(dev(C), gp, 3, 91, 1000, 2)
    b.step(30)
    for k in range(3):
        ga = g.GA(dev(C), gp, seed=91 + k)
        ga.step(30)
        lab, L, gen = ga.best()
        ga.close()
        lb, Lb, gb = b.best(k)
        np.testing.assert_array_equal(lb, lab)
        assert Lb == L and gb == gen == 30
    b.close()


def test_island_arguments(g, orc):
    p = synth.small16()
    C = orc.pearson(p.R)
    gp, _ = _params(g, orc, 16)
    for bad in [dict(islands=1, every=2, m=1), dict(islands=3, every=0, m=1),
                dict(islands=3, every=2, m=5), dict(islands=3, every=2, m=0)]:
        with pytest.raises(g.GpgaError):
            g.Batch.islands(dev(C), gp, bad["islands"], 1, bad["every"], bad["m"])
