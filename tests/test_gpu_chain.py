"""Checkpoint/resume of a libhmc chain on the GPU: four trajectories straight through against
two, a checkpoint, a new context loading it and two more. The fields must agree bit for bit and
the JSONL records (except the measured phase times) must be identical."""

import json

import numpy as np
import pytest
import torch

from paper_2204_14241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COUPLINGS = dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5, u=1.0, c=3.0)


def context():
    from paper_2204_14241_gb300.hmc import Context
    return Context(8, 8, solver="mixed", nrhs_max=2, cg_tol=1e-10, initial_guess=3, **COUPLINGS)


def test_checkpoint_resume_is_bit_identical(tmp_path):
    from paper_2204_14241_gb300.chain import Chain
    phi0 = I.gaussian_field(60, 8, 8) * 0.6
    sig = torch.ones((3, 8, 8, 8), dtype=torch.float64, device="cuda")
    logs = {}
    ctx_a = context()
    a = Chain(ctx_a, torch.from_numpy(phi0.copy()).cuda(), sig, 0.05, n_max=6, nrhs=2, seed=5,
              log=str(tmp_path / "a.jsonl"))
    a.run(4)
    ctx_b = context()
    b = Chain(ctx_b, torch.from_numpy(phi0.copy()).cuda(), sig, 0.05, n_max=6, nrhs=2, seed=5,
              log=str(tmp_path / "b.jsonl"))
    b.run(2)
    b.save(tmp_path / "ck.npz")
    ctx_b.close()
    ctx_c = context()
    c = Chain.load(tmp_path / "ck.npz", ctx_c, log=str(tmp_path / "b.jsonl"))
    c.run(2)
    assert torch.equal(a.phi, c.phi)
    for name in ("a", "b"):
        logs[name] = [json.loads(x) for x in open(tmp_path / f"{name}.jsonl")]
    for ra, rb in zip(logs["a"], logs["b"]):
        ra.pop("phase_ms")
        rb.pop("phase_ms")
        assert ra == rb
    assert len(logs["a"]) == len(logs["b"]) == 4
    assert all(r["status"] == 0 and len(r["solve_iterations"]) == r["n_leap"] + 1 for r in logs["a"])
