"""Writes the FP64 oracle's diagnostics time series that the long-window GPU
tests compare with (tests/test_gpu_series.py).

Only the oracle (oracle/) and the seeded input generator (stgv_inputs.py) are
used: no value here comes from the CUDA path. Each series is a stratified
Taylor-Green run (Eq. 20 initial field, Section 2.4 parameter mapping, Eq. 19)
advanced by the oracle's two-lattice FP64 update (Eqs. 5-18), with the
diagnostics of Eqs. 22-26 sampled every `every` steps.

Usage: python tests/golden/make_oracle_series.py [name ...]
(no name: every series below; the output is tests/golden/<name>.txt)
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import stgv_inputs as inputs  # noqa: E402
from oracle import oracle  # noqa: E402

# name: (n, (qf, qg), forcing, Re, Fr, Sc, U0, steps, every, seed, noise_amp)
SERIES = {
    # the n/Re of the 256^3 Re 800 workload (same tau_f) at 64^3, run to t ~ 20
    # convective times (254.6 steps each): a laminar, strongly stratified decay
    # whose dissipation oscillates early (acoustic and internal waves)
    "stgv64_re200_fr01_sc": (64, (27, 19), "sc", 200.0, 0.1, 1.0, 0.04, 5100, 25, 1, 1e-3),
    # the paper's parameters (Section 2.4: Re0 1600, Sc 0.7, Ma 0.1 so U0 = 0.0577,
    # Fr0 1) at 64^3 to t ~ 30 (176.5 steps per convective time): the
    # turbulent breakdown and its dissipation peaks (Section 3.3)
    "stgv64_paper_re1600_fr1_sc": (64, (27, 19), "sc", 1600.0, 1.0, 0.7, 0.0577, 5310, 18, 1, 1e-3),
}
# the 128^3 workload: both stencil pairs x {Guo, Shan-Chen} x Fr {0.5, 0.1}, Re 400,
# 5000 steps with the diagnostics every 50 steps
for _q in ((19, 7), (27, 19)):
    for _f in ("guo", "sc"):
        for _fr in (0.5, 0.1):
            SERIES[f"c1_128_q{_q[0]}q{_q[1]}_{_f}_fr{_fr}"] = (128, _q, _f, 400.0, _fr, 1.0, 0.04, 5000, 50, 1, 1e-3)

COLUMNS = ("step", "Ek", "Ep", "eps_k", "eps_p", "eps_k_curl", "mass_f", "mass_g", "mom_x", "mom_y",
           "mom_z", "umax")


def path_of(name: str) -> str:
    return os.path.join(HERE, name + ".txt")


def write(name: str) -> str:
    n, (qf, qg), forcing, Re, Fr, Sc, U0, steps, every, seed, amp = SERIES[name]
    p = oracle.params_from_physics(n, qf, qg, forcing, Re, Fr, Sc, U0)
    sim = oracle.OracleSim(p)
    sim.init_fields(*inputs.tgv_fields(n, U0, seed=seed, noise_amp=amp))
    rows = []
    t0 = time.time()
    for k in range(steps // every + 1):
        if k:
            sim.step(every)
        d = sim.diagnostics()
        rows.append([d[c] for c in COLUMNS])
    sim.close()
    out = path_of(name)
    with open(out + ".tmp", "w") as fh:
        fh.write(f"# FP64 oracle series {name}: n={n} D3Q{qf}xD3Q{qg} forcing={forcing} Re={Re} Fr={Fr} "
                 f"Sc={Sc} U0={U0} steps={steps} every={every}\n")
        fh.write(f"# initial field: Eq. 20 + {amp} U0 SplitMix64 noise (seed {seed}); "
                 f"written by tests/golden/make_oracle_series.py ({oracle.num_threads()} threads, "
                 f"{time.time() - t0:.0f} s)\n")
        fh.write("# " + " ".join(COLUMNS) + "\n")
        for r in rows:
            fh.write(" ".join([str(int(r[0]))] + [f"{v:.17g}" for v in r[1:]]) + "\n")
    os.replace(out + ".tmp", out)
    return out


def read(name: str) -> list[dict]:
    rows = []
    with open(path_of(name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            vals = line.split()
            d = {c: float(v) for c, v in zip(COLUMNS, vals)}
            d["step"] = int(vals[0])
            rows.append(d)
    return rows


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(SERIES)):
        print(write(name))
