"""Photometric bundle adjustment on the GPU (gsdf_energy_ba_step) against the oracle's step.

Same inputs as the energy tests: keyframes of the room, a voxel list fused by the oracle with psi
and g rounded to FP32, the oracle's visibility.  Bars:
  * mean colours within 1e-4 (FP32 bilinear samples of FP32 images, averaged);
  * residual counts exact (the same index-path decisions);
  * normal equations: each photometric term carries ~1e-4 relative FP32 error (a projection good
    to ~1e-4 px moves the bilinear weights), so |dH_ij| <= 1e-3 sqrt(H_ii H_jj),
    |db_i| <= 1e-3 sqrt(H_ii E), |dE| <= 1e-4 E;
  * updated poses within 1e-4 (rad / m) and psi within 1e-5 m of the oracle's, in lockstep.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_energy import _case, _dev, _pack  # noqa: E402


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


@pytest.fixture(scope="module")
def small():
    return _case(4, I.TINY_160, 0.02)


@pytest.fixture(scope="module")
def full():
    return _case(10, I.KINECT_640, 0.01)


def _setup(G, case, poses=None):
    ks, m, psi, g, rho = case
    poses = ks.poses if poses is None else poses
    nu = O.visibility(m, psi.astype(np.float64), g.astype(np.float64), ks.voxel_size, ks.cam, poses, ks.depths)
    en = G.Energy(_dev(m), ks.voxel_size, G.intrinsics(ks.cam), _dev(ks.rgbs), _dev(ks.depths))
    return en, nu


def _gpu_step(G, en, psi, g, poses, nu, lam, damping, flags):
    F = len(poses)
    psi_t, P = _dev(psi), _dev(np.stack(poses).astype(np.float64))
    rho = torch.empty((len(psi), 3), dtype=torch.float32, device="cuda")
    stats = torch.zeros((F, G.TRACK_STATS_BYTES), dtype=torch.uint8, device="cuda")
    en.ba_step(psi_t, _dev(g), rho, P, _dev(_pack(nu)), lam, damping, flags, stats)
    st = [G.track_stats_from_bytes(x) for x in stats.cpu().numpy()]
    return psi_t.cpu().numpy(), rho.cpu().numpy(), [x for x in P.cpu().numpy()], st


def _assert_normal(st, ost):
    assert st.n_valid == ost.n_valid
    Ho, Hg = O.stats_H(ost), O.stats_H(st)
    d = np.sqrt(np.maximum(np.diag(Ho), 0))
    assert np.all(np.abs(Hg - Ho) <= 1e-3 * np.outer(d, d) + 1e-12), np.max(np.abs(Hg - Ho) / (np.outer(d, d) + 1e-30))
    btol = 1e-3 * np.sqrt(np.diag(Ho) * ost.energy) + 1e-12
    assert np.all(np.abs(np.array(st.b) - np.array(ost.b)) <= btol)
    assert st.energy == pytest.approx(ost.energy, rel=1e-4)


@pytest.mark.parametrize("lam", [0.0, 100.0])
def test_evaluation_matches_oracle_small(G, small, lam):
    ks, m, psi, g, _ = small
    en, nu = _setup(G, small)
    _, rho, _, st = _gpu_step(G, en, psi, g, ks.poses, nu, lam, 0.0, 0)
    _, orho, _, ost, _, _ = O.ba_step(m, psi.astype(np.float64), g.astype(np.float64), ks.voxel_size, ks.cam,
                                      ks.poses, ks.rgbs, ks.depths, nu, lam, 0.0, 0)
    assert np.max(np.abs(rho - orho)) <= 1e-4
    for i in range(len(ks.poses)):
        _assert_normal(st[i], ost[i])
    en.close()


def test_evaluation_matches_oracle_full_size(G, full):
    ks, m, psi, g, _ = full
    en, nu = _setup(G, full)
    _, rho, _, st = _gpu_step(G, en, psi, g, ks.poses, nu, 100.0, 0.0, 0)
    _, orho, _, ost, _, _ = O.ba_step(m, psi.astype(np.float64), g.astype(np.float64), ks.voxel_size, ks.cam,
                                      ks.poses, ks.rgbs, ks.depths, nu, 100.0, 0.0, 0)
    assert np.max(np.abs(rho - orho)) <= 1e-4
    for i in range(len(ks.poses)):
        _assert_normal(st[i], ost[i])
    en.close()


def test_pose_and_psi_updates_in_lockstep(G, small):
    ks, m, psi, g, _ = small
    rng = np.random.default_rng(8)
    poses = [T.copy() for T in ks.poses]
    for i in range(1, len(poses)):
        poses[i] = I.perturb_pose(poses[i], rng, 0.3, 0.003)
    en, nu = _setup(G, small, poses)
    err0 = np.mean([np.linalg.norm(poses[i][:3, 3] - ks.poses[i][:3, 3]) for i in range(1, len(poses))])
    flags = G.GSDF_BA_POSES
    for it in range(6):
        _, _, gposes, st = _gpu_step(G, en, psi, g, poses, nu, 100.0, 1e-4, flags)
        _, _, poses, ost, _, _ = O.ba_step(m, psi.astype(np.float64), g.astype(np.float64), ks.voxel_size, ks.cam,
                                           poses, ks.rgbs, ks.depths, nu, 100.0, 1e-4, O.BA_POSES)
        for i in range(len(poses)):
            assert st[i].status == ost[i].status == 0
            assert np.abs(gposes[i] - poses[i]).max() < 1e-4, (it, i)
    err = np.mean([np.linalg.norm(poses[i][:3, 3] - ks.poses[i][:3, 3]) for i in range(1, len(poses))])
    assert err < 0.2 * err0
    # one damped psi step on a perturbed map
    psi_p = (psi + rng.normal(0, 0.002, size=len(psi))).astype(np.float32)
    gpsi, _, _, _ = _gpu_step(G, en, psi_p, g, ks.poses, nu, 100.0, 1.0, G.GSDF_BA_PSI)
    opsi, _, _, _, _, _ = O.ba_step(m, psi_p.astype(np.float64), g.astype(np.float64), ks.voxel_size, ks.cam,
                                    ks.poses, ks.rgbs, ks.depths, nu, 100.0, 1.0, O.BA_PSI)
    moved = np.abs(opsi - psi_p) > 0
    assert moved.sum() > 1000
    assert np.max(np.abs(gpsi - opsi)) <= 1e-5
    en.close()


def test_arguments(G, small):
    ks, m, psi, g, _ = small
    en, nu = _setup(G, small)
    L = G.load_library()
    assert G.gsdf_energy_ba_step(en.e, 0, 0, 0, 0, 0, 1.0, 0.0, 1) == G.GSDF_ERR_INVALID_ARG
    P = _dev(np.stack(ks.poses))
    assert G.gsdf_energy_ba_step(en.e, _dev(psi).data_ptr(), _dev(g).data_ptr(), 0, P.data_ptr(), 0, 1.0, 0.0,
                                 8) == G.GSDF_ERR_INVALID_ARG
    assert L.gsdf_energy_ba_step(None, None, None, None, None, None, 0.0, 0.0, 0, None) == G.GSDF_ERR_INVALID_ARG
    en.close()
