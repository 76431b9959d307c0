"""The allocation-free potential solve (GPU).

ehdlb_potential_noalloc serves callers that cannot call cudaMalloc: code
inside an allocator or memory-pool callback, processes whose device memory
another runtime owns, loops that must not risk an allocation's implicit
synchronisation.  It keeps every intermediate in one fixed-size device array
of the library.  Checked here against the context solver (the existing entry
point) and against the oracle, each on two calls in a row, since the second
call finds the first one's contents in the shared array.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2501_04920_gb300 import ehdlb, workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def noalloc(torch, nx, ny, p, phi, q, K):
    """Two calls in a row on the current stream; each returns (status, r, psi, Ex, Ey)."""
    dev = torch.device("cuda", 0)
    phi_d = torch.tensor(phi, dtype=torch.float64, device=dev)
    q_d = torch.tensor(q, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    calls = []
    for _ in range(2):
        out = [torch.full((ny, nx), float("nan"), dtype=torch.float64, device=dev) for _ in range(3)]
        status, r = ehdlb.ehdlb_potential_noalloc(nx, ny, p, phi_d.data_ptr(), q_d.data_ptr(), K,
                                                  out[0].data_ptr(), out[1].data_ptr(),
                                                  out[2].data_ptr(), stream)
        torch.cuda.synchronize(dev)
        calls.append((status, r, *[t.cpu().numpy() for t in out]))
    return calls


def test_noalloc_potential_matches_the_context_solver_on_two_calls():
    torch = pytest.importorskip("torch")
    nx, ny, K = 96, 80, 257
    prm = workloads.droplet64()
    prm.update(xc=(nx - 1) / 2, yc=(ny - 1) / 2, R=20.0, eps_r=4.0, psi_anode=2.0,
               init_sweeps_fixed=K)
    # the existing entry point: set_params solves the initial potential with
    # q = 0 in K sweeps; its snapshot holds phi, psi and E.  A second context
    # stops one sweep earlier, which gives the residual of the last sweep.
    lat = ehdlb.Lattice(nx, ny, prm, precision=ehdlb.FP64)
    ref = lat.fields(["phi", "psi", "Ex", "Ey"])
    lat.close()
    lat = ehdlb.Lattice(nx, ny, dict(prm, init_sweeps_fixed=K - 1), precision=ehdlb.FP64)
    before = lat.fields(["psi"])["psi"]
    lat.close()
    r_ref = np.sqrt(np.sum((ref["psi"] - before) ** 2) / np.sum(ref["psi"] ** 2))
    p = ehdlb.ehdlb_params_default(prm)
    for call, (status, r, psi, Ex, Ey) in enumerate(noalloc(torch, nx, ny, p, ref["phi"],
                                                            np.zeros((ny, nx)), K)):
        assert status == ehdlb.OK, call
        assert abs(r - r_ref) <= 1e-8 * r_ref, (call, r, r_ref)
        for name, v in (("psi", psi), ("Ex", Ex), ("Ey", Ey)):
            assert rel_linf(v, ref[name]) <= FP64_TOL, (call, name)


def test_noalloc_potential_with_charge_and_side_walls_matches_the_oracle():
    # a non-square lattice closed by side walls, the potential started from
    # zero, and a net charge q = sum p - sum n that varies in x and y: the
    # oracle takes one step with K sweeps from that state, and its snapshot
    # holds psi and E after the sweeps and the phi and q they used
    torch = pytest.importorskip("torch")
    nx, ny, K = 52, 37, 40
    prm = workloads.droplet64()
    prm.update(xc=20.0, yc=(ny - 1) / 2, R=9.0, eps_r=4.0, Kq=0.05, psi_anode=1.5,
               psi_cathode=-0.5, side_walls=1, init_psi_zero=1, init_sweeps_fixed=0)
    orc = oracle.Oracle(nx, ny, prm)
    s = orc.state()
    yy, xx = np.mgrid[0:ny, 0:nx]
    cp = 1.0 + 0.3 * np.sin(2 * np.pi * xx / nx) * np.cos(np.pi * yy / ny)
    cm = 1.0 - 0.2 * np.cos(2 * np.pi * (xx + yy) / nx)
    w5 = np.array([1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6])
    s[:, :, 18:23] = cp[..., None] * w5
    s[:, :, 23:28] = cm[..., None] * w5
    assert np.all(s[:, :, 28:33] == 0.0)       # the potential starts from zero
    orc.set_state(s)
    _, res, _ = orc.step(1, forced=[K])
    ref = orc.fields()
    assert np.max(np.abs(ref["q"])) > 0.3
    p = ehdlb.ehdlb_params_default(prm)
    for call, (status, r, psi, Ex, Ey) in enumerate(noalloc(torch, nx, ny, p, ref["phi"], ref["q"], K)):
        assert status == ehdlb.OK, call
        assert abs(r - res[0]) <= 1e-8 * res[0], (call, r, res[0])
        for name, v in (("psi", psi), ("Ex", Ex), ("Ey", Ey)):
            assert rel_linf(v, ref[name]) <= FP64_TOL, (call, name, rel_linf(v, ref[name]))


def test_noalloc_rejects_lattices_above_its_maximum():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    p = ehdlb.ehdlb_params_default()
    a = torch.zeros(4, dtype=torch.float64, device=dev)
    n = 257  # 257 x 257 > EHDLB_NOALLOC_MAX_NODES
    status, _ = ehdlb.ehdlb_potential_noalloc(n, n, p, a.data_ptr(), a.data_ptr(), 1,
                                              a.data_ptr(), a.data_ptr(), a.data_ptr())
    assert status == ehdlb.EINVAL
