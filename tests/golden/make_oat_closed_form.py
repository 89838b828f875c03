"""Writes oat_closed_form.json: the exact one-axis-twisting moment of Sec. II.B.

<S^x(t)> = (N/2) cos^(N-1)(t) (Eq. 13) for an all-+x initial state, sampled at
the GSE-TDVP1 step times dt, 2dt, ...  Run parameters follow the paper's
Delta t = 0.025 setting (tau = dt, k = 3, eps_K = eps_M = 1e-4, eps = 0),
with N reduced so the dense checks stay small.
"""
import json
import math
import os

N, DT, STEPS = 12, 0.025, 10
out = dict(source="Sec. II.B, Eq. 13 (closed form); parameters of the Delta t = 0.025 run",
           n_sites=N, dt=DT, steps=STEPS, k=3, eps_k=1e-4, eps_m=1e-4,
           sx=[0.5 * N * math.cos(DT * s) ** (N - 1) for s in range(1, STEPS + 1)],
           tol_sx=2e-3)
json.dump(out, open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                 "oat_closed_form.json"), "w"), indent=1)
