"""Pins of the oracle's two-relaxation-time (TRT) collision (Sec. II.A, TRT
paragraph, Eq. magic-parameter), against facts that do not come from the oracle:

- with Lambda = (tau - 1/2)^2 the two rates are equal and TRT is BGK;
- on one periodic node (streaming is the identity) an even non-conserved mode
  decays by (1 - omega+) per step and an odd mode without momentum by
  (1 - omega-), with omega- from Eq. magic-parameter;
- collision and Guo forcing conserve mass and add exactly F of momentum per node;
- with Lambda = 3/16 half-way bounce-back puts the wall of a body-force channel
  exactly half-way, at any tau: the steady profile is the parabola of the
  Navier-Stokes solution to round-off (the property the paper recalls for this
  Lambda). BGK at large tau misses it, so the check has teeth.
"""
import numpy as np
import pytest

import oracle
from paper_2009_04604_gb300 import workloads as W


def _omega_minus(tau, magic):
    # Eq. magic-parameter with omega+ = 1/tau, solved for omega-
    return 1.0 / (0.5 + magic / (tau - 0.5))


@pytest.mark.parametrize("bc", [oracle.BC_ELIBB_F, oracle.BC_ELIBB_FQ, oracle.BC_BFL, oracle.BC_HWBB,
                                oracle.BC_ELIBB_U, oracle.BC_ELIBB_UQ])
def test_trt_with_equal_rates_is_bgk(oracle_lib, bc):
    dims = (7, 6, 5)
    tau = 0.83
    flags, q, uw, uw1, tag = W.random_geometry(dims, seed=9, Q=19)
    F = (1e-5, -2e-5, 3e-6)
    pb = oracle.params(oracle.D3Q19, dims, tau, bc=bc, force=F)
    pt = oracle.params(oracle.D3Q19, dims, tau, bc=bc, force=F, collision=oracle.COLL_TRT,
                       magic=(tau - 0.5) ** 2)
    f = oracle.init_eq(pb, flags)
    rng = np.random.default_rng(4)
    f = f * (1.0 + 0.05 * rng.standard_normal(f.shape))
    fb, ft = f, f
    for _ in range(3):
        fb = oracle.step(pb, flags, fb, q, uw, uw1)
        ft = oracle.step(pt, flags, ft, q, uw, uw1)
    assert np.abs(fb - ft).max() < 1e-14


@pytest.mark.parametrize("tau,magic", [(0.8, 3.0 / 16.0), (0.6, 0.25), (1.7, 1.0 / 12.0)])
def test_trt_relaxes_even_and_odd_modes_at_their_rates(oracle_lib, tau, magic):
    p = oracle.params(oracle.D2Q9, (1, 1, 1), tau, collision=oracle.COLL_TRT, magic=magic)
    c, w, _ = oracle.lattice(oracle.D2Q9)
    cx, cy = c[:, 0].astype(float), c[:, 1].astype(float)
    c2 = cx ** 2 + cy ** 2
    even = cx ** 2 - cy ** 2           # no mass, no momentum (even in c)
    odd = cx * (3.0 * c2 - 5.0)        # no mass (odd), no momentum: sum_i odd_i c_i = 0
    assert abs(even.sum()) < 1e-15 and np.abs(odd @ c).max() < 1e-15
    flags = np.zeros(1, np.uint8)
    feq = oracle.init_eq(p, flags)[0]  # rho = 1, u = 0
    eps_e, eps_o = 1e-3, 2e-3
    f = (feq + eps_e * even + eps_o * odd)[None, :]
    fo = oracle.step(p, flags, f)[0]
    wp, wm = 1.0 / tau, _omega_minus(tau, magic)
    expect = feq + (1.0 - wp) * eps_e * even + (1.0 - wm) * eps_o * odd
    assert np.abs(fo - expect).max() < 1e-15


@pytest.mark.parametrize("lat,dims", [(oracle.D2Q9, (8, 6, 1)), (oracle.D3Q19, (5, 4, 6)),
                                      (oracle.D3Q27, (4, 5, 3))])
def test_trt_mass_and_momentum_balance(oracle_lib, lat, dims):
    rng = np.random.default_rng(6)
    F = np.array([2e-5, -1e-5, 0.0 if lat == oracle.D2Q9 else 3e-5])
    p = oracle.params(lat, dims, 0.9, force=F, collision=oracle.COLL_TRT, magic=3.0 / 16.0)
    N = p.nx * p.ny * p.nz
    flags = np.zeros(N, np.uint8)
    c, w, _ = oracle.lattice(lat)
    f = w[None, :] * (1.0 + 0.05 * rng.standard_normal((N, len(w))))
    m0, j0 = f.sum(), (f @ c).sum(0)
    for _ in range(10):
        f = oracle.step(p, flags, f)
    assert abs(f.sum() - m0) / m0 < 1e-14
    np.testing.assert_allclose((f @ c).sum(0) - j0, 10 * N * F, atol=1e-13)


def _channel(tau, collision, magic=3.0 / 16.0, H=12, g=1e-6):
    """Body-force channel between half-way bounce-back walls (solid rows y = 0 and
    H + 1): returns the steady velocity of rows 1..H and the Navier-Stokes parabola
    with walls at y = 1/2 and H + 1/2."""
    ny = H + 2
    p = oracle.params(oracle.D2Q9, (1, ny, 1), tau, bc=oracle.BC_HWBB, force=(g, 0.0, 0.0),
                      collision=collision, magic=magic)
    flags = np.zeros(ny, np.uint8)
    flags[0] = flags[-1] = oracle.SOLID
    s = oracle.Sim(p, flags)
    nu = (tau - 0.5) / 3.0
    steps = int(40 * H * H / (np.pi ** 2 * nu)) + 200
    s.run(steps)
    u = s.macros()[1][1:H + 1, 0]
    y = np.arange(1, H + 1, dtype=float)
    return u, g / (2.0 * nu) * (y - 0.5) * (H + 0.5 - y)


@pytest.mark.parametrize("tau", [0.6, 1.0, 3.0])
def test_trt_magic_3_16_puts_bounce_back_wall_half_way(oracle_lib, tau):
    u, uth = _channel(tau, oracle.COLL_TRT)
    assert np.abs(u - uth).max() / uth.max() < 1e-9


def test_bgk_bounce_back_wall_moves_with_tau(oracle_lib):
    u, uth = _channel(3.0, oracle.COLL_BGK)
    assert np.abs(u - uth).max() / uth.max() > 1e-2
