"""Parity report: the error of every likelihood form and of the Pearson prelude
against the FP64 oracle, per workload, as a markdown table (the figures the
tests bound by |dL| <= 1e-4 + 1e-6 |L| and max |dC| <= 1e-6).

    python tests/parity_report.py > profiles/parity_errors_by_form.md

Needs a GPU and the built library; the expected values come from oracle/ only.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1403_4099_gb300 import gpga, synth  # noqa: E402

FORMS = {"plain (FP32)": gpga.FORM_PLAIN, "tensor (BF16 hi+lo, tcgen05)": gpga.FORM_TENSOR,
         "gather (int32 fixed point)": gpga.FORM_GATHER}


def populations(truth, P, rng):
    N = truth.shape[0]
    return {
        "uniform labels": synth.random_labels(rng, P, N),
        "few labels (N/12)": synth.random_labels(rng, P, N, K=max(2, N // 12)),
        "converged (planted, 5% redrawn)": synth.perturbed_population(rng, truth, P, 0.05),
    }


def main():
    import torch
    oracle.build()
    gpga.lib()
    work = [("small16 (N=16, T=500)", synth.small16(), 64),
            ("n100 (N=100, T=2000)", synth.n100(), 1024),
            ("n500 (N=500, T=5000)", synth.n500(), 4096)]
    print("# Likelihood and correlation errors against the FP64 oracle\n")
    print("Command: `python tests/parity_report.py` (1 GB300). Same seeded inputs on both "
          "sides; the oracle's C is the input of every GPU score. Bar per individual: "
          "|dL| <= 1e-4 + 1e-6 |L|.\n")
    print("| workload | population | form | P | max abs dL | p99 abs dL | max dL / bar | mean L |")
    print("|---|---|---|---:|---:|---:|---:|---:|")
    corr_rows = []
    for wname, pl, P in work:
        C = oracle.pearson(pl.R)
        Cg = gpga.cluster_corr(torch.from_numpy(pl.R).cuda())
        torch.cuda.synchronize()
        corr_rows.append((wname, float(np.abs(Cg.cpu().numpy() - C).max())))
        rng = np.random.default_rng(7)
        for pname, pop in populations(pl.truth, P, rng).items():
            t0 = time.perf_counter()
            ref = oracle.loglik_batch(pop, C)
            _ = time.perf_counter() - t0
            lab = torch.from_numpy(np.ascontiguousarray(pop, np.int32)).cuda()
            Cd = torch.from_numpy(C).cuda()
            for fname, form in FORMS.items():
                L = gpga.ga_score(lab, Cd, form=form)
                torch.cuda.synchronize()
                got = L.cpu().numpy()
                err = np.abs(got - ref)
                bar = 1e-4 + 1e-6 * np.abs(ref)
                print(f"| {wname} | {pname} | {fname} | {P} | {err.max():.2e} | "
                      f"{np.percentile(err, 99):.2e} | {(err / bar).max():.3f} | "
                      f"{ref.mean():.4g} |")
    print("\n| workload | max abs dC (cluster_corr vs oracle Pearson) |")
    print("|---|---:|")
    for wname, e in corr_rows:
        print(f"| {wname} | {e:.2e} |")


if __name__ == "__main__":
    main()
