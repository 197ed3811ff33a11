"""Pins of the oracle's photometric bundle-adjustment step (Sec. 4.2, Eqs. rgb_cost, mean_color,
rgb_cost_pose) -- the Gauss-Newton terms of the decoupled per-keyframe energies with the mean
colour held fixed, optionally plus lambda times the geometric term of Eq. (tracking).

* With rho = the step's mean colours, the step's b_i and psi terms are half the gradient of the
  energy oracle (a separately written adjoint): 2 b_i = dE/dxi_i, 2 psi_b = dE/dpsi, and the
  keyframe energies add up to E.
* On single (voxel, keyframe) pairs, H_i = sum_c J_c J_c^T and psi_H = sum_c (dI_c/dpsi)^2 with J_c
  from central differences of the sampled colour I_c (read off the energy's d/drho at rho = 0)
  under scipy's expm.
* Pose-only iterations pull perturbed keyframe poses back toward the truth when the geometric
  term anchors them to the map (lambda = 100 = sigma_I^2 / sigma_d^2 for colour noise ~0.01 and
  depth noise ~1 mm; on this small, smoothly textured problem the photometric term alone leaves
  the cameras' common placement weakly constrained); a psi-only step on a perturbed map lowers
  the energy.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I
from test_oracle_energy_pins import _safe_nu, _twist


@pytest.fixture(scope="module")
def setup():
    ks = I.keyframes(seed=2, n_keyframes=4, stride=10, cam=I.TINY_160, voxel_size=0.02)
    m_ = O.OracleMap(O.params(ks.voxel_size, huber_delta=1e9))
    for i in range(len(ks.poses)):
        m_.integrate(ks.depths[i], ks.cam, ks.poses[i])
    ex = m_.extract()
    nu = O.visibility(ex["m"], ex["psi"], ex["g"], ks.voxel_size, ks.cam, ks.poses, ks.depths)
    return ks, ex, nu


def _step(ks, ex, nu, lam, flags=0, poses=None, psi=None, damping=0.0):
    return O.ba_step(ex["m"], ex["psi"] if psi is None else psi, ex["g"], ks.voxel_size, ks.cam,
                     ks.poses if poses is None else poses, ks.rgbs, ks.depths, nu, lam, damping, flags)


@pytest.mark.parametrize("lam", [0.0, 0.5])
def test_gradient_terms_equal_half_the_energy_gradient(setup, lam):
    ks, ex, nu = setup
    _, rho, _, st, hp, hb = _step(ks, ex, nu, lam)
    E, dpsi, _, drho, dxi, _ = O.energy(ex["m"], ex["psi"], ex["g"], rho, ks.voxel_size, ks.cam, ks.poses, ks.rgbs,
                                        ks.depths, nu, lam)
    assert np.max(np.abs(drho)) < 1e-9  # rho is the minimiser in rho (Eq. mean_color)
    for i in range(len(ks.poses)):
        assert np.allclose(2 * np.array(st[i].b), dxi[i], rtol=1e-9, atol=1e-9 * np.abs(dxi).max())
    assert np.allclose(2 * hb, dpsi, rtol=1e-9, atol=1e-9 * np.abs(dpsi).max())
    assert sum(s.energy for s in st) == pytest.approx(E[0], rel=1e-12)
    assert np.all(hp >= 0) and np.sum(hp > 0) > 500


def test_normal_equations_on_single_pairs(setup):
    ks, ex, nu = setup
    safe = _safe_nu(ks, ex, nu, margin=0.05)
    rng = np.random.default_rng(3)
    pairs = np.argwhere(safe)
    zero_rho = np.zeros((len(ex["psi"]), 3))

    def colour(nu1, poses, psi):
        _, _, _, drho, _, _ = O.energy(ex["m"], psi, ex["g"], zero_rho, ks.voxel_size, ks.cam, poses, ks.rgbs,
                                       ks.depths, nu1, 0.0)
        return -0.5 * drho  # I_c of the one counted pair, zero elsewhere

    for i, j in pairs[rng.choice(len(pairs), 6, replace=False)]:
        nu1 = np.zeros_like(nu)
        nu1[i, j] = 1
        _, _, _, st, hp, _ = _step(ks, ex, nu1, 0.0)
        h = 1e-7
        Jc = np.zeros((3, 6))
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Pp = [scipy.linalg.expm(_twist(e)) @ T if q == i else T for q, T in enumerate(ks.poses)]
            Pm = [scipy.linalg.expm(_twist(-e)) @ T if q == i else T for q, T in enumerate(ks.poses)]
            Jc[:, k] = (colour(nu1, Pp, ex["psi"])[j] - colour(nu1, Pm, ex["psi"])[j]) / (2 * h)
        H = O.stats_H(st[i])
        assert np.allclose(H, Jc.T @ Jc, rtol=1e-4, atol=1e-6 * np.abs(H).max())
        hq = 1e-7
        pp, pm = ex["psi"].copy(), ex["psi"].copy()
        pp[j] += hq
        pm[j] -= hq
        jpsi = (colour(nu1, ks.poses, pp)[j] - colour(nu1, ks.poses, pm)[j]) / (2 * hq)
        assert hp[j] == pytest.approx(np.sum(jpsi**2), rel=1e-4)
        assert st[i].n_valid == 3


def test_pose_only_iterations_recover_perturbed_poses(setup):
    ks, ex, nu = setup
    rng = np.random.default_rng(8)
    poses = [T.copy() for T in ks.poses]
    for i in range(1, len(poses)):
        poses[i] = I.perturb_pose(poses[i], rng, 0.3, 0.003)
    err0 = [np.linalg.norm(poses[i][:3, 3] - ks.poses[i][:3, 3]) for i in range(1, len(poses))]
    nu_p = O.visibility(ex["m"], ex["psi"], ex["g"], ks.voxel_size, ks.cam, poses, ks.depths)
    energies = []
    for _ in range(8):
        _, _, poses, st, _, _ = _step(ks, ex, nu_p, 100.0, O.BA_POSES, poses=poses, damping=1e-4)
        energies.append(sum(s.energy for s in st))
        assert all(s.status == 0 for s in st)
    err = [np.linalg.norm(poses[i][:3, 3] - ks.poses[i][:3, 3]) for i in range(1, len(poses))]
    assert energies[-1] < 0.2 * energies[0]
    assert np.mean(err) < 0.2 * np.mean(err0), (err0, err)
    assert np.linalg.norm(poses[0][:3, 3] - ks.poses[0][:3, 3]) < 5e-3  # the unperturbed keyframe stays


def test_psi_only_step_lowers_the_energy(setup):
    ks, ex, nu = setup
    rng = np.random.default_rng(9)
    psi = ex["psi"] + rng.normal(0, 0.002, size=len(ex["psi"]))
    psi1, rho, _, st, _, _ = _step(ks, ex, nu, 0.0, O.BA_PSI, psi=psi, damping=1.0)
    E0 = sum(s.energy for s in st)
    E1 = O.energy(ex["m"], psi1, ex["g"], rho, ks.voxel_size, ks.cam, ks.poses, ks.rgbs, ks.depths, nu, 0.0,
                  grad=False)[0]
    assert E1 < E0
