"""The serving loop on the GPU (needs a GB300): a served case's result is the
result of the same case run alone for the same number of steps."""
import pytest

from paper_2501_04920_gb300 import ehdlb
from paper_2501_04920_gb300.serve import Case, Server, serve_one_by_one

pytestmark = pytest.mark.gpu


def test_served_cases_match_their_runs_alone():
    cases = [Case(t=0.0, nx=64 + 64 * (i % 2), ny=128, d_mm=0.5 + 0.4 * i, dpsi_kV=1.0 + i, eps_r=[0.5, 2.0, 4.0, 1.0][i],
                  mu_r=[2.0, 0.5, 1.0, 2.0][i], key=i) for i in range(4)]
    # room for two cases at a time: the others wait and take the freed memory
    budget = 2 * ehdlb.ehdlb_batch_footprint(ehdlb.FP32, 128, 128) + (1 << 20)
    b = ehdlb.Batch(budget, 20)
    res = Server(b, check_every=40, max_steps=200, tol=2e-7).run(cases)
    b.close()
    assert sorted(r.key for r in res) == [0, 1, 2, 3]
    for r in res:
        c = cases[r.key]
        lat = ehdlb.Lattice(c.nx, c.ny, c.params(20))
        lat.step(r.steps)
        assert lat.deformation() == r.D
        lat.close()
    alone = {r.key: r for r in serve_one_by_one(cases, check_every=40, max_steps=200, tol=2e-7)}
    for r in res:
        assert alone[r.key].steps == r.steps and alone[r.key].D == r.D
