"""The -DHMC_BOUNDS build of libhmc: index checks in the D operator, the force and the strip
operator record failed checks in device error words instead of accessing memory. A clean run of
the operators, a solve and a trajectory through that build must record nothing and give the same
results as the oracle (run in a subprocess that loads the bounds library through HMC_LIBRARY)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2204_14241_gb300 import hmc as H, inputs as I
assert H.LIB_PATH.endswith("libhmc_bounds.so"), H.LIB_PATH
C = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5, u=1.0, c=3.0)
out = {}
for L, Nt in ((16, 8), (12, 6)):
    ctx = H.Context(L, Nt, solver="mixed", nrhs_max=2, cg_tol=1e-10, initial_guess=2, **C)
    phi = torch.from_numpy(I.gaussian_field(3, L, Nt) * 0.6).cuda()
    x = torch.from_numpy(I.fermion_noise(4, 2, L, Nt)).cuda()
    y32 = ctx.apply_MdagM(phi.float(), x.to(torch.complex64))
    yD = ctx.apply_M(phi, x)
    F, spf, sb, st = ctx.force(phi, x, precond=False)
    o = ctx.trajectory([phi], [torch.ones_like(phi)], 0.05, 3, nrhs=2, precond=False, seed=1, counter=0)
    out[f"{L}x{Nt}"] = {"y32": y32.cpu().numpy().astype(np.complex128).ravel()[:64].tolist(),
                        "yD_abs_sum": float(yD.abs().sum()), "spf": spf, "status": o["status"]}
    ctx.close()
torch.cuda.synchronize()
w, enabled = H.bounds_status()
print(json.dumps({"word": w, "enabled": enabled, "runs": {k: {"status": v["status"]} for k, v in out.items()}}))
"""


def test_bounds_build_records_nothing_on_clean_runs():
    from paper_2204_14241_gb300 import build
    lib = os.path.join(ROOT, "paper_2204_14241_gb300", "libhmc_bounds.so")
    if not os.path.exists(lib):
        build.build(variant="_bounds")
    env = dict(os.environ, HMC_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["enabled"] is True
    assert res["word"] == 0, res
    assert all(v["status"] == 0 for v in res["runs"].values())
