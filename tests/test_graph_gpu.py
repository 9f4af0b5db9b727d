"""The CUDA-graph replay of the float32 LOBPCG iteration (the launches
before and after the SpMM captured once per handle and preconditioner, the
timed SpMM between them) against direct launches (LOBPCG_GRAPH=0, in a
child process): the same Ritz values iteration by iteration, to float32
rounding, for the diagonal, block-Jacobi and FOM forms."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

CODE = r"""
import json, sys, numpy as np, torch, synth
import paper_2109_00485_gb300 as pkg
pkg.load()
stream = torch.cuda.Stream()          # a created stream: the legacy default stream cannot be captured
A = synth.tile_matrix(3000, 60, seed=4)
A = synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))
X0 = synth.initial_guess(A, 8, seed=1001, fp32=True)
out = {}
for pc in ("diag", "bjacobi", "fom"):
    h = pkg.from_csr(A, k=8, nev=5, tol=1e-6, maxiter=1000, precond=pc, polish_fp64=1, stream=stream)
    th = []
    t, _ = h.iterate(1, X0=X0)
    th.append([float(v) for v in t])
    for _ in range(6):
        t, _ = h.iterate(1)
        th.append([float(v) for v in t])
    X, ev, rs, st = h.solve(X0)
    h.destroy()
    out[pc] = {"theta": th, "ev": [float(v) for v in ev], "conv": int(st["converged"])}
print(json.dumps(out))
"""


def _run(graph: str):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, LOBPCG_GRAPH=graph, PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", CODE], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_graph_replay_matches_direct_launches():
    g, d = _run("1"), _run("0")
    for pc in ("diag", "bjacobi", "fom"):
        tg, td = np.array(g[pc]["theta"]), np.array(d[pc]["theta"])
        # the SpMM adds transposed contributions in no fixed order, so the
        # two runs differ by float32 rounding that grows slowly with the steps
        assert np.all(np.abs(tg - td) <= 1e-4 * np.maximum(np.abs(td), 1.0)), (pc, tg - td)
        assert g[pc]["conv"] == 1 and d[pc]["conv"] == 1
        assert np.allclose(g[pc]["ev"], d[pc]["ev"], rtol=1e-8, atol=1e-9)
