"""The allocation-free potential solve against the context solver (GPU).

ehdlb_potential_noalloc serves callers that cannot call cudaMalloc (allocator
callbacks, processes whose device memory another runtime owns, loops that must
not risk an allocation's implicit synchronisation); it keeps every
intermediate in one fixed-size device array of the library.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2501_04920_gb300 import ehdlb, workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_noalloc_potential_matches_the_context_solver_on_two_calls():
    torch = pytest.importorskip("torch")
    nx, ny, K = 96, 80, 257
    prm = workloads.droplet64()
    prm.update(xc=(nx - 1) / 2, yc=(ny - 1) / 2, R=20.0, eps_r=4.0, psi_anode=2.0,
               init_sweeps_fixed=K)
    # the existing entry point: set_params solves the initial potential with
    # q = 0 in K sweeps; its snapshot holds phi, psi and E
    lat = ehdlb.Lattice(nx, ny, prm, precision=ehdlb.FP64)
    ref = lat.fields(["phi", "psi", "Ex", "Ey"])
    p = ehdlb.ehdlb_params_default(prm)
    dev = torch.device("cuda", 0)
    phi = torch.tensor(ref["phi"], dtype=torch.float64, device=dev)
    q = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        out = [torch.full((ny, nx), float("nan"), dtype=torch.float64, device=dev) for _ in range(3)]
        status, r = ehdlb.ehdlb_potential_noalloc(nx, ny, p, phi.data_ptr(), q.data_ptr(), K,
                                                  out[0].data_ptr(), out[1].data_ptr(),
                                                  out[2].data_ptr(), stream)
        torch.cuda.synchronize(dev)
        assert status == ehdlb.OK, call
        assert np.isfinite(r) and r < 1e-2, r
        for name, t in zip(("psi", "Ex", "Ey"), out):
            assert rel_linf(t.cpu().numpy(), ref[name]) <= FP64_TOL, (call, name)
    lat.close()


def test_noalloc_rejects_lattices_above_its_maximum():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    p = ehdlb.ehdlb_params_default()
    a = torch.zeros(4, dtype=torch.float64, device=dev)
    n = 257  # 257 x 257 > EHDLB_NOALLOC_MAX_NODES
    status, _ = ehdlb.ehdlb_potential_noalloc(n, n, p, a.data_ptr(), a.data_ptr(), 1,
                                              a.data_ptr(), a.data_ptr(), a.data_ptr())
    assert status == ehdlb.EINVAL
