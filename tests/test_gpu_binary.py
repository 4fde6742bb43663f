"""The paper's binary orbit test (Sec. 4) as a short run: two point masses (GM =
0.01 each, separation 0.15) deposited by CIC onto an AMR grid that follows them,
kick-drift-kick leapfrog with a fixed step over one orbit.  Bounds: the first
acceleration against the two-body value (CIC and FMM discretisation only), the
energy and angular momentum of the orbit, the separation, and the centre of
mass (the setup is point-symmetric about the box centre)."""
import numpy as np
import pytest

from paper_2607_19489_b300 import binary

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lmax", [6, 7, 8])
def test_one_orbit_conserves(lmax):
    b = binary.Binary(lmin=6, lmax=lmax, p=6, precision="mixed")
    a = b.accel()
    sep = b.x[0] - b.x[1]
    a_two_body = -b.m[1] * sep / np.linalg.norm(sep) ** 3
    assert np.linalg.norm(a[0] - a_two_body) / np.linalg.norm(a_two_body) < 0.02
    assert np.linalg.norm(a[0] + a[1]) / np.linalg.norm(a[0]) < 0.02   # equal and opposite
    period = 2 * np.pi / b.omega
    d = b.run(period, period / 64)
    assert abs(d["dE_over_E0"]) < 5e-3, d
    assert abs(d["dL_over_L0"]) < 5e-3, d
    assert abs(d["dr_over_r0"]) < 0.03, d
    assert d["com_drift"] < 1e-4, d
