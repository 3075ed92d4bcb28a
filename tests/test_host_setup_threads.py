"""The host setup gives the same hierarchy whatever the number of OpenMP
threads (CPU only).

The setup's parallel steps (transposes split into chunks of source rows,
the PMIS sweeps, the symmetrised and sparsified Galerkin products, the
assembly of the AMGR reduced operator) each write a result that does not
depend on how the rows are shared out, and every sum keeps its serial
order.  The problem here is large enough (1.4M nonzeros in A_inn) for the
chunked transposes; every matrix the library exposes is compared byte for
byte between 1 and 4 threads.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import hashlib, json
import numpy as np
import paper_2407_05930_gb300 as amg
from synth import gaussian_logk

N, s = (96, 64, 64), 1
P = amg.Problem.structured(N, 1.5, gaussian_logk(N, s, seed=5, corr=4.0), s).setup(host_only=1, amgr=1)
out = {}
for l in range(P.num_levels()):
    for w in ("A", "P", "G"):
        if l == P.num_levels() - 1 and w != "A":
            continue
        rp, ci, v, shape = P.level_matrix(l, w)
        out["L%d%s" % (l, w)] = hashlib.sha256(rp.tobytes() + ci.tobytes() + v.tobytes()).hexdigest()
    out["L%domega" % l] = P.level_info(l)["omega"]
info = P.amgr_info()
out["cf"] = hashlib.sha256(info["cf"].tobytes()).hexdigest()
for w in ("P", "Ac"):
    rp, ci, v, shape = P.amgr_matrix(w)
    out["amgr" + w] = hashlib.sha256(rp.tobytes() + ci.tobytes() + v.tobytes()).hexdigest()
out["nnz"] = int(P.level_info(0)["nnz_A"])
print("RESULT " + json.dumps(out))
"""


def _run(threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", _CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_hierarchy_is_independent_of_the_thread_count():
    one, four = _run(1), _run(4)
    assert one["nnz"] >= 1 << 20  # the chunked transpose path
    assert one == four
