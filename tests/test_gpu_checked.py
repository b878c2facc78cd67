"""The checked build (build.py, checked=True; -DBEM_CHECKED=1).

Its kernels compare every global index they write -- partial-sum slots,
per-point arrays, rows of the near-pair prefix table, assembled-matrix
entries -- and every near-pair record they read against the capacity of the
buffer it indexes, skip an access that would fall outside, and flag it; the
call then returns an error.  This test runs every entry point that launches
the far and near kernels through the checked library in a child process (the
library is chosen when it is loaded, so it cannot share this process) on
small cases that span several point tiles and element chunks with a ragged
tail, and requires that nothing was flagged and that the results equal the
release build's.  No access is made to go out of range on purpose: the
checks only record, and a fault is never provoked.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_1606_03743_gb300 as bem
import synth

out = {"version": bem.bem_version()}
res = {}
mesh = synth.plate_mesh(seed=1, n=24)            # 1728 elements: several chunks
pts = synth.plate_points(seed=2, n=5000)         # several 128-point tiles, ragged tail
gp = synth.plate_points(seed=3, n=700)
for prec, table in ((0, False), (1, False), (1, True)):
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec, node_table=table) as m:
        phi, E = m.eval(pts)
        res[f"eval_{prec}_{int(table)}"] = np.concatenate([phi[:, None], E], axis=1)
        if not table:
            res[f"grad_{prec}"] = m.eval_grad(gp)
            res[f"asm_{prec}"] = m.assemble(synth.collocation_points(mesh)[:300])
coef = np.zeros((mesh.n, 3))
coef[:, 0] = mesh.sigma
coef[:, 1] = 0.3
with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=1) as m:
    m.set_sigma_linear(coef)
    phi, E = m.eval(pts)
    res["linear"] = np.concatenate([phi[:, None], E], axis=1)
import torch
dev = torch.device("cuda", 0)
with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=1) as m:
    tp = torch.from_numpy(pts).to(dev)
    phi = torch.empty(len(pts), dtype=torch.float64, device=dev)
    E = torch.empty((len(pts), 3), dtype=torch.float64, device=dev)
    bem.bem_eval_noalloc(m.handle, tp, phi, E)
    torch.cuda.synchronize()
    res["noalloc"] = np.concatenate([phi.cpu().numpy()[:, None], E.cpu().numpy()], axis=1)
    with bem.Server(m, max_points_per_tick=2048) as srv:
        tickets = [srv.submit(pts[a:b]) for a, b in ((0, 100), (100, 3100), (3100, 5000))]
        parts = [srv.wait(t, timeout=120) for t in tickets]
    res["server"] = np.concatenate([np.concatenate([p[:, None], e], axis=1) for p, e in parts])
np.savez(OUT, **res)
print(json.dumps(out))
"""


def _release_results(bem):
    mesh = synth.plate_mesh(seed=1, n=24)
    pts = synth.plate_points(seed=2, n=5000)
    gp = synth.plate_points(seed=3, n=700)
    res = {}
    for prec, table in ((0, False), (1, False), (1, True)):
        with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec, node_table=table) as m:
            phi, E = m.eval(pts)
            res[f"eval_{prec}_{int(table)}"] = np.concatenate([phi[:, None], E], axis=1)
            if not table:
                res[f"grad_{prec}"] = m.eval_grad(gp)
                res[f"asm_{prec}"] = m.assemble(synth.collocation_points(mesh)[:300])
    coef = np.zeros((mesh.n, 3))
    coef[:, 0] = mesh.sigma
    coef[:, 1] = 0.3
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=1) as m:
        m.set_sigma_linear(coef)
        phi, E = m.eval(pts)
        res["linear"] = np.concatenate([phi[:, None], E], axis=1)
    return res


def test_checked_build_flags_nothing_and_matches_release(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_03743_gb300 as bem
    bem.load_library()
    out = tmp_path / "checked.npz"
    env = dict(os.environ, BEM_CHECKED="1")
    code = f"ROOT = {ROOT!r}\nOUT = {str(out)!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    info = json.loads(r.stdout.strip().splitlines()[-1])
    assert "checked" in info["version"]
    assert "checked" not in bem.bem_version()
    got = dict(np.load(out))
    ref = _release_results(bem)
    # FP64 and mixed paths: the same arithmetic in both builds; the checks add
    # comparisons only, so the values agree to the last few bits
    for k, v in ref.items():
        tol = 1e-13 if k in ("eval_0_0", "grad_0", "asm_0") else 1e-7
        scale = np.abs(v).max()
        assert np.abs(got[k] - v).max() <= tol * scale, k
    # no-allocation and serving paths (mixed precision) against the release bem_eval
    for k in ("noalloc", "server"):
        v = ref["eval_1_0"]
        assert np.abs(got[k] - v).max() <= 1e-7 * np.abs(v).max(), k
