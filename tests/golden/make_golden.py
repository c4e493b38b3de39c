"""Writes oracle_tiny.json: oracle outputs on tiny seeded cases (calls only oracle/):
the cell-centred path, with source bases, with oversampled edges and faces, and the
nodal Galerkin variant.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.galerkin_oracle import NodalOracle  # noqa: E402
from oracle.msfv_oracle import Oracle  # noqa: E402
from paper_1707_07598_gb300 import workloads as W  # noqa: E402

CASES = [dict(n=[12, 8], c=4, ns=2, nr=6, seed=3, corr=0.3),
         dict(n=[6, 6, 6], c=3, ns=2, nr=5, seed=4, corr=0.3),
         dict(n=[12, 8], c=4, ns=2, nr=6, seed=5, corr=0.3, sb=True),
         dict(n=[8, 8, 8], c=4, ns=2, nr=7, seed=6, corr=0.3, sb=True),
         dict(n=[12, 8], c=4, ns=2, nr=6, seed=7, corr=0.3, nodal=True),
         dict(n=[6, 6, 6], c=3, ns=2, nr=5, seed=8, corr=0.3, nodal=True),
         dict(n=[12, 8], c=4, ns=2, nr=6, seed=9, corr=0.3, ov=2),
         dict(n=[8, 8, 8], c=4, ns=2, nr=7, seed=10, corr=0.3, ov=1)]

out = []
for case in CASES:
    prob = W.make_problem(tuple(case['n']), case['c'], case['ns'], case['nr'],
                          seed=case['seed'], top_layer=False,
                          source_bases=case.get('sb', False), nodal=case.get('nodal', False),
                          oversample=case.get('ov', 0))
    m = W.gaussian_random_field(prob.n, case['corr'], case['seed'] + 2)
    o = NodalOracle(prob) if case.get('nodal') else Oracle(prob)
    st = o.forward(m)
    d_obs = st['d'] * 1.02 + 0.01
    phi, g = o.misfit_gradient(st, d_obs)
    out.append(dict(case, d=st['d'].tolist(), d_obs=d_obs.tolist(), grad=g.tolist(), phi=phi))
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json"), "w") as f:
    json.dump(out, f)
print("wrote", len(out), "cases")
