"""The error of every likelihood form and of the Pearson prelude against the
FP64 oracle, per workload and population regime, through the C-ABI: every
individual within |dL| <= 1e-4 + 1e-6 |L| and max |dC| <= 1e-6 (asserted).
With PARITY_TABLE_OUT=<path> in the environment the figures are also written
there as a markdown table, e.g.

    PARITY_TABLE_OUT=/tmp/parity_errors_by_form.md \\
        python -m pytest tests/test_gpu_parity_table.py -m gpu -q

The expected values come from oracle/ only."""
import os

import numpy as np
import pytest

from paper_1403_4099_gb300 import synth

pytestmark = pytest.mark.gpu

FORMS = (("plain (FP32)", 0), ("tensor (BF16 hi+lo, tcgen05)", 1), ("gather (int32 fixed point)", 2))


def _populations(truth, P, rng):
    N = truth.shape[0]
    return {
        "uniform labels": synth.random_labels(rng, P, N),
        "few labels (N/12)": synth.random_labels(rng, P, N, K=max(2, N // 12)),
        "converged (planted, 5% redrawn)": synth.perturbed_population(rng, truth, P, 0.05),
    }


def test_parity_table(orc):
    import torch
    from paper_1403_4099_gb300 import build, gpga
    build.build()
    work = [("small16 (N=16, T=500)", synth.small16(), 64),
            ("n100 (N=100, T=2000)", synth.n100(), 1024),
            ("n500 (N=500, T=5000)", synth.n500(), 4096)]
    rows, corr_rows, worst = [], [], 0.0
    for wname, pl, P in work:
        C = orc.pearson(pl.R)
        Cg = gpga.cluster_corr(torch.from_numpy(pl.R).cuda())
        torch.cuda.synchronize()
        ec = float(np.abs(Cg.cpu().numpy() - C).max())
        corr_rows.append((wname, ec))
        assert ec <= 1e-6, (wname, ec)
        rng = np.random.default_rng(7)
        Cd = torch.from_numpy(C).cuda()
        for pname, pop in _populations(pl.truth, P, rng).items():
            ref = orc.loglik_batch(pop, C)
            lab = torch.from_numpy(np.ascontiguousarray(pop, np.int32)).cuda()
            bar = 1e-4 + 1e-6 * np.abs(ref)
            for fname, form in FORMS:
                L = gpga.ga_score(lab, Cd, form=form)
                torch.cuda.synchronize()
                err = np.abs(L.cpu().numpy() - ref)
                worst = max(worst, float((err / bar).max()))
                rows.append(f"| {wname} | {pname} | {fname} | {P} | {err.max():.2e} | "
                            f"{np.percentile(err, 99):.2e} | {(err / bar).max():.3f} | "
                            f"{ref.mean():.4g} |")
    out = os.environ.get("PARITY_TABLE_OUT")
    if out:
        with open(out, "w") as f:
            f.write("# Likelihood and correlation errors against the FP64 oracle\n\n")
            f.write(f"Command: `PARITY_TABLE_OUT={out} python -m "
                    "pytest tests/test_gpu_parity_table.py -m gpu -q` (1 GB300). Same seeded "
                    "inputs on both sides; the oracle's C is the input of every GPU score. Bar "
                    "per individual: |dL| <= 1e-4 + 1e-6 |L|.\n\n")
            f.write("| workload | population | form | P | max abs dL | p99 abs dL | "
                    "max dL / bar | mean L |\n|---|---|---|---:|---:|---:|---:|---:|\n")
            f.write("\n".join(rows) + "\n\n| workload | max abs dC (cluster_corr vs oracle "
                    "Pearson) |\n|---|---:|\n")
            f.write("\n".join(f"| {w} | {e:.2e} |" for w, e in corr_rows) + "\n")
    assert worst <= 1.0, worst
