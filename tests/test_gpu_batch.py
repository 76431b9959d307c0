"""Batches of uneven lattices stepped by the persistent kernels (needs a GB300).

A case in a batch runs the per-block code of the single-lattice kernels on
the same inputs, so its fields must equal those of the same case stepped
alone, bit for bit; the deformation factor computed on the device must equal
Eq. 63 evaluated by the oracle on the same phi field.
"""
import numpy as np
import pytest

import oracle
from paper_2501_04920_gb300 import ehdlb

pytestmark = pytest.mark.gpu

SWEEPS = 20


def case_params(nx, ny, d_mm, dpsi, eps_r, mu_r):
    p = ehdlb.ehdlb_params_from_physical(nx, ny, d_mm, dpsi, eps_r, mu_r)
    p.sweeps_min = p.sweeps_max = SWEEPS
    return p


CASES = [(128, 192, 1.0, 2.0, 2.0, 0.5), (192, 128, 2.0, 1.0, 0.5, 2.0),
         (64, 64, 0.5, 3.0, 4.0, 1.0), (256, 320, 1.5, 4.0, 1.0, 2.0)]


def alone(nx, ny, p, steps, precision):
    lat = ehdlb.Lattice(nx, ny, p, precision=precision)
    lat.step(steps)
    f = lat.fields()
    d = lat.deformation()
    lat.close()
    return f, d


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", [ehdlb.FP32, ehdlb.FP16S])
def test_batched_cases_equal_the_same_cases_alone(precision, shape):
    # tile shape 1: the sweeps in shared memory; 2: in registers
    b = ehdlb.Batch(2 << 30, SWEEPS, precision=precision)
    ehdlb.ehdlb_batch_set_tuning(b.b, -1, shape, -1)
    ids = [b.add(nx, ny, case_params(nx, ny, *c)) for nx, ny, *c in CASES]
    steps = 30
    b.step(steps - 7)
    _, st = b.step(7)
    assert st.cases == len(CASES) and st.unstable_cases == 0
    D = b.deformation(ids)
    for cid, (nx, ny, *c), dd in zip(ids, CASES, D):
        ref, d_alone = alone(nx, ny, case_params(nx, ny, *c), steps, precision)
        got = b.fields(cid)
        for k in ehdlb.FIELDS:
            assert np.array_equal(got[k], ref[k]), (nx, ny, k)
        assert dd == d_alone
    b.close()


# Uneven cases of the physical mapping (Sec. 3; R = nx / 5), each against the
# oracle run alone on the same parameters, at the FP32 parity tolerance.
ORACLE_CASES = [(96, 128, 1.2, 2.5, 2.0, 0.5), (128, 96, 0.8, 1.5, 0.5, 2.0), (64, 112, 1.6, 3.5, 4.0, 1.0)]


def test_batched_uneven_cases_match_the_oracle():
    from test_gpu_parity import FP32_TOL, FP32_U_TOL, field_errors
    steps = 40
    b = ehdlb.Batch(1 << 30, SWEEPS)
    ids = [b.add(nx, ny, case_params(nx, ny, *c)) for nx, ny, *c in ORACLE_CASES]
    _, st = b.step(steps)
    assert st.cases == len(ORACLE_CASES) and st.unstable_cases == 0
    for cid, (nx, ny, *c) in zip(ids, ORACLE_CASES):
        prm = oracle.params_from_physical(nx, ny, *c)
        prm.update(sweeps_min=SWEEPS, sweeps_max=SWEEPS)
        orc = oracle.Oracle(nx, ny, prm)
        orc.step(steps)
        err = field_errors(b.fields(cid), orc.fields())
        bad = {k: v for k, v in err.items() if k in ("phi", "psi", "q", "cp", "cm") and not v <= FP32_TOL}
        if not err["u"] <= FP32_U_TOL:
            bad["u"] = err["u"]
        assert not bad, (nx, ny, bad, err)
    b.close()


def test_cases_join_and_leave_without_disturbing_the_others():
    b = ehdlb.Batch(2 << 30, SWEEPS)
    (nx0, ny0, *c0), (nx1, ny1, *c1), (nx2, ny2, *c2) = CASES[:3]
    a = b.add(nx0, ny0, case_params(nx0, ny0, *c0))
    gone = b.add(nx1, ny1, case_params(nx1, ny1, *c1))
    b.step(10)
    b.remove(gone)
    late = b.add(nx2, ny2, case_params(nx2, ny2, *c2))
    b.step(12)
    ref_a, _ = alone(nx0, ny0, case_params(nx0, ny0, *c0), 22, ehdlb.FP32)
    ref_late, _ = alone(nx2, ny2, case_params(nx2, ny2, *c2), 12, ehdlb.FP32)
    fa, fl = b.fields(a), b.fields(late)
    for k in ehdlb.FIELDS:
        assert np.array_equal(fa[k], ref_a[k]), k
        assert np.array_equal(fl[k], ref_late[k]), k
    b.close()


def test_admission_by_footprint():
    one = ehdlb.ehdlb_batch_footprint(ehdlb.FP32, 256, 256)
    b = ehdlb.Batch(int(2.5 * one), SWEEPS)
    p = case_params(256, 256, 1.0, 2.0, 2.0, 2.0)
    first, second = b.add(256, 256, p), b.add(256, 256, p)
    assert first is not None and second is not None
    assert b.add(256, 256, p) is None                 # no room for a third
    n, used, cap = b.info()
    assert n == 2 and used <= cap
    b.remove(first)
    assert b.add(256, 256, p) is not None             # its memory is reused
    assert ehdlb.ehdlb_batch_footprint(ehdlb.FP16S, 256, 256) < one
    b.close()


def test_batch_rejects_cases_it_does_not_take():
    b = ehdlb.Batch(1 << 30, SWEEPS)
    with pytest.raises(ehdlb.EhdlbError):
        b.add(100, 64, case_params(100, 64, 1.0, 1.0, 2.0, 2.0))        # nx not a multiple of 8
    p = case_params(64, 64, 1.0, 1.0, 2.0, 2.0)
    p.sweeps_max = p.sweeps_min = 5
    with pytest.raises(ehdlb.EhdlbError):
        b.add(64, 64, p)                                                 # other sweep count
    with pytest.raises(ehdlb.EhdlbError):
        b.step(1)                                                        # empty batch
    b.close()


@pytest.mark.parametrize("nx,ny", [(64, 96), (128, 192), (300, 520), (2048, 2048)])
def test_device_deformation_is_eq63_of_the_fields(nx, ny):
    # one slice of the device sums, a few, slices ending inside rows, the most slices
    lat = ehdlb.Lattice(nx, ny, case_params(nx, ny, 1.0, 4.0, 0.5, 5.0))
    lat.step(40)
    phi = lat.fields(["phi"])["phi"]
    assert abs(lat.deformation() - oracle.deformation(phi)) <= 1e-12
    lat.close()


def test_reporting_captures_the_asked_fields_and_returns_D():
    nx, ny = 128, 192
    lat = ehdlb.Lattice(nx, ny, case_params(nx, ny, 1.0, 4.0, 0.5, 5.0))
    lat.step(20)
    phi_bit = 1 << ehdlb.FIELDS.index("phi")
    ehdlb.ehdlb_set_reporting(lat.ctx, phi_bit, 1)
    _, st = lat.step(20)
    # D read back with the step's counters is D of the captured phi
    assert st.deformation == lat.deformation()
    assert abs(st.deformation - oracle.deformation(lat.fields(["phi"])["phi"])) <= 1e-12
    with pytest.raises(ehdlb.EhdlbError):
        lat.fields(["ux"])                      # not captured by the last step
    ehdlb.ehdlb_set_reporting(lat.ctx, 0, 1)    # D alone still captures phi
    _, st = lat.step(1)
    assert st.deformation == lat.deformation()
    ehdlb.ehdlb_set_reporting(lat.ctx, (1 << len(ehdlb.FIELDS)) - 1, 0)
    _, st = lat.step(1)
    assert np.isnan(st.deformation)
    assert set(lat.fields()) >= {"phi", "ux", "q"}
    with pytest.raises(ehdlb.EhdlbError):
        ehdlb.ehdlb_set_reporting(lat.ctx, 1 << len(ehdlb.FIELDS), 0)
    with pytest.raises(ehdlb.EhdlbError):
        ehdlb.ehdlb_set_reporting(lat.ctx, phi_bit, 2)
    lat.close()


def test_autotuner_picks_a_valid_schedule():
    b = ehdlb.Batch(1 << 30, SWEEPS)
    for nx, ny, *c in CASES[:2]:
        b.add(nx, ny, case_params(nx, ny, *c))
    spl, shape, ms = b.autotune(3)
    assert spl in (3, 4, 5) and shape in (0, 1, 2) and ms > 0
    _, st = b.step(2)
    assert st.sweeps_per_launch == spl and st.tile_shape == shape
    b.close()
