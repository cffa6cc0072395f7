"""Host logic of the chain driver (paper_2204_14241_gb300.chain) with a stand-in context whose
trajectory is a deterministic function of (phi, seed, counter, n_leap): Philox counters follow
the trajectory index, n_leap jitter is reproducible, the JSONL records are complete, and a chain
saved and resumed reproduces the uninterrupted chain exactly."""

import json

import numpy as np
import torch

from paper_2204_14241_gb300.chain import Chain


class StandInContext:
    device = torch.device("cpu")

    def trajectory(self, phis, sigmas, eps, n_leap, nrhs, precond, seed, counter, check):
        g = np.random.default_rng([seed, counter, n_leap])
        step = torch.from_numpy(g.standard_normal(tuple(phis[0].shape))) * eps
        dH = float(g.standard_normal())
        acc = bool(g.random() < min(1.0, np.exp(-dH)))
        if acc:
            phis[0].add_(step * (1.0 + 0.1 * phis[0].abs().mean()))
        self.last = n_leap
        return {"status": 0, "dH": [dH], "accepted": [acc], "energies": [[1.0, 2.0, 3.0, 1.5, 2.5, 3.5]],
                "cg_iterations": [7 * (n_leap + 1)], "max_true_resid": [1e-11]}

    def trajectory_stats(self, chain):
        n = self.last + 1
        return {"n_solves": n, "reliable_updates": 2 * n, "iterations": [7] * n, "true_resid": [1e-11] * n,
                "phase_ms": {"solve": 1.0, "force": 0.1, "metric": 0.2, "other": 0.05}}


def make(log, **kw):
    phi = torch.from_numpy(np.random.default_rng(0).standard_normal((3, 4, 6, 6)))
    return Chain(StandInContext(), phi, torch.ones_like(phi), 0.05, nrhs=2, seed=11, log=log, **kw)


def test_resume_reproduces_the_uninterrupted_chain(tmp_path):
    for kw in ({"n_leap": 5}, {"n_max": 6, "jitter_seed": 3}):
        full_log, part_log = tmp_path / "full.jsonl", tmp_path / "part.jsonl"
        full_log.unlink(missing_ok=True)
        part_log.unlink(missing_ok=True)
        a = make(str(full_log), **kw)
        a.run(6)
        b = make(str(part_log), **kw)
        b.run(2)
        b.save(tmp_path / "ck.npz")
        c = Chain.load(tmp_path / "ck.npz", StandInContext(), log=str(part_log), device="cpu")
        assert c.index == 2 and c.eps == 0.05 and c.seed == 11 and c.nrhs == 2
        c.run(4)
        assert torch.equal(a.phi, c.phi) and a.accepted == c.accepted and a.index == c.index == 6
        full = [json.loads(x) for x in open(full_log)]
        part = [json.loads(x) for x in open(part_log)]
        assert full == part and [r["index"] for r in full] == list(range(6))
        for r in full:
            assert r["solve_iterations"] == [7] * (r["n_leap"] + 1)
            assert set(r["phase_ms"]) == {"solve", "force", "metric", "other"}
            assert set(r["energies"]) == {"kinetic_start", "S_B_start", "S_PF_start", "kinetic_end", "S_B_end",
                                          "S_PF_end"}


def test_jitter_draws_cover_one_to_n_max():
    c = make(None, n_max=4, jitter_seed=9)
    draws = [c.trajectory_length(i) for i in range(200)]
    assert set(draws) == {1, 2, 3, 4}
    assert draws == [make(None, n_max=4, jitter_seed=9).trajectory_length(i) for i in range(200)]
