"""Temperature recovery of the FP32 modes at single nodes (Eq. e7), away
from any step: populations stored in FP32 (random equilibria of Eqs.
e16-e18 at up to Mach 30, each population perturbed by about 1e-5
relative) are set as the level, and the moments the library returns are
compared with the same Eqs. e4, e5, e7 evaluated in FP64 by the oracle on
exactly those FP32 values.

The model's constants are chosen exactly representable in FP32 (c1 = 33,
diagonal component c2 / sqrt(2) = 56.5, eta0 = 40, b = 5), so the two sides
differ in arithmetic only.  Each mode's error is bounded by what its own
arithmetic rounds (u = 2^-24, e = rho b T the internal energy, E the total
energy moment, w_i = |v_i - u|^2 + eta_i^2):
  * fp32_tdf, fp32_t64: the nine terms f_i w_i are formed around u (an
    error in u enters e only at second order, since sum f_i (v_i - u) = 0),
    each w_i with a few FP32 roundings, and summed exactly enough (double-
    float, or FP64): |e error| <= 4 u sum |f_i w_i| + 4 u e;
  * fp32 (the same terms summed in plain FP32): 8 more roundings of the
    running sum, |e error| <= 12 u sum |f_i w_i| + 4 u e;
  * fp32_cons (e = E - rho u^2 in FP32, E = sum f_i q_i with q_i = |v_i|^2
    + eta_i^2): |e error| <= 8 u sum |f_i| q_i + 2 rho |u| du + 4 u (E + e),
    du the bound on u below.
rho = sum f_i and u = (sum f_i v_i) / rho are FP32 sums in every mode:
|rho error| <= 8 u sum |f_i|, |u error| <= du = 8 u (sum |f_i| |v_i| +
|u| sum |f_i|) / rho + 4 u |u|.
With the KT equilibrium some moving populations are negative at high Mach,
so these absolute sums exceed rho, rho |u| and e by up to 10^4 here: the
bounds say how much each mode may lose, and the test checks that none loses
more (an error in the method's arithmetic, a wrong term or sign, would
miss them by orders of magnitude)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_0706_0405_gb300 import lbm
from paper_0706_0405_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C1, D, ETA0, B = 33.0, 56.5, 40.0, 5.0
U = 2.0 ** -24


def _problem(nx=64, ny=16):
    return W.uniform(nx, ny, (1.0, 0.0, 0.0, 1.0), c1=C1, c2=D * math.sqrt(2.0), eta0=ETA0, dx=0.01,
                     b=B)


@pytest.fixture(scope="module")
def level():
    """FP32 populations (9, ny, nx), the oracle's FP64 moments of them, and
    per node sum |f_i w_i| and E (FP64)."""
    p = _problem()
    rng = np.random.Generator(np.random.PCG64(2024))
    n = p.nx * p.ny
    rho = np.exp(rng.uniform(math.log(0.1), math.log(10.0), n))
    T = np.exp(rng.uniform(math.log(0.05), math.log(2.0), n))
    mach = rng.uniform(0.0, 30.0, n)
    ang = rng.uniform(0.0, 2.0 * math.pi, n)
    speed = np.minimum(mach * np.sqrt(1.4 * T), 25.0)  # below c1
    ux, uy = speed * np.cos(ang), speed * np.sin(ang)
    vx, vy = oracle.velocities(p.c1, p.c2)
    eta2 = np.zeros(9)
    eta2[0] = p.eta0 ** 2
    f = np.empty((9, n))
    ref = np.empty((4, n))
    sabs, E, qabs, fabs, vabs = (np.empty(n) for _ in range(5))
    for k in range(n):
        f9 = oracle.feq(p, rho[k], ux[k], uy[k], T[k]) * (1.0 + 1e-5 * rng.standard_normal(9))
        f9 = f9.astype(np.float32).astype(np.float64)
        f[:, k] = f9
        ref[:, k] = oracle.moments(p, f9)
        w = (vx - ref[1, k]) ** 2 + (vy - ref[2, k]) ** 2 + eta2
        q = vx ** 2 + vy ** 2 + eta2
        sabs[k] = np.sum(np.abs(f9 * w))
        E[k] = np.sum(f9 * q)
        qabs[k] = np.sum(np.abs(f9) * q)
        fabs[k] = np.sum(np.abs(f9))
        vabs[k] = np.sum(np.abs(f9) * np.hypot(vx, vy))
    assert np.all(ref[3] > 0.0)
    speed = np.hypot(ref[1], ref[2])
    du = 8.0 * U * (vabs + speed * fabs) / ref[0] + 4.0 * U * speed
    bounds = {"sabs": sabs, "E": E, "qabs": qabs, "rho": 8.0 * U * fabs, "du": du}
    return p, f.reshape(9, p.ny, p.nx).astype(np.float32), ref, bounds


def _gpu_moments(p, prec, f32):
    with lbm.Lattice(p, prec) as lat:
        lat.set_f(torch.from_numpy(f32).cuda())
        return np.stack([t.double().cpu().numpy().ravel() for t in lat.moments()])


def _energy_error(got, ref):
    """|e error| of the returned T: b rho |T - T_ref|."""
    return B * ref[0] * np.abs(got[3] - ref[3])


def _check_rho_u(got, ref, bd):
    assert (np.abs(got[0] - ref[0]) / bd["rho"]).max() <= 1.0
    assert (np.abs(got[1] - ref[1]) / bd["du"]).max() <= 1.0
    assert (np.abs(got[2] - ref[2]) / bd["du"]).max() <= 1.0


@pytest.mark.parametrize("prec,k_sum", [("fp32_tdf", 4.0), ("fp32_t64", 4.0), ("fp32", 12.0)])
def test_internal_energy_modes_within_their_rounding_bound(level, prec, k_sum):
    p, f32, ref, bd = level
    got = _gpu_moments(p, prec, f32)
    _check_rho_u(got, ref, bd)
    e = B * ref[0] * ref[3]
    bound = k_sum * U * bd["sabs"] + 4.0 * U * e
    ratio = _energy_error(got, ref) / bound
    assert ratio.max() <= 1.0, (prec, ratio.max())


def test_total_energy_mode_within_its_rounding_bound(level):
    p, f32, ref, bd = level
    got = _gpu_moments(p, "fp32_cons", f32)
    _check_rho_u(got, ref, bd)
    e = B * ref[0] * ref[3]
    speed = np.hypot(ref[1], ref[2])
    bound = 8.0 * U * bd["qabs"] + 2.0 * ref[0] * speed * bd["du"] + 4.0 * U * (bd["E"] + e)
    ratio = _energy_error(got, ref) / bound
    assert ratio.max() <= 1.0, ratio.max()


def test_double_float_sum_is_at_least_as_accurate_as_the_plain_fp32_sum(level):
    """The double-float and FP64 sums agree with each other to the rounding
    of the terms; the plain FP32 sum of the same terms is no closer to the
    FP64 moments than they are (summed over the nodes)."""
    p, f32, ref, bd = level
    tdf = _energy_error(_gpu_moments(p, "fp32_tdf", f32), ref)
    t64 = _energy_error(_gpu_moments(p, "fp32_t64", f32), ref)
    plain = _energy_error(_gpu_moments(p, "fp32", f32), ref)
    assert tdf.sum() <= 1.5 * t64.sum() + 1e-30 and t64.sum() <= 1.5 * tdf.sum() + 1e-30
    assert tdf.sum() <= plain.sum()
