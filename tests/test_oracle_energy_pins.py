"""Pins of the oracle's photometric + geometric voxel energy (Sec. 4.2) and its gradient.

* Central finite differences of the oracle's own energy: psi, g and rho entries (photometric and
  geometric terms), the keyframe poses under a left perturbation by scipy's matrix exponential,
  and the 12 entries of each pose matrix (both terms).  The energy is piecewise smooth in the
  pose: the bilinear cell and the geometric term's voxel are discrete choices.  The pose
  differences therefore run on a visibility subset whose points stay 1e-2 px away from any cell
  boundary and on depth images whose back-projected points stay 1e-3 v_s away from any voxel
  boundary, so that no choice changes within the step.
* The left-perturbation gradient equals the matrix gradient contracted with the generators
  [e_k]x T of SE(3) (two separately written formulas).
* The geometric pose gradient against the tracking reduction, a separately written code path:
  with a Huber threshold too large to clip, b = sum J r, so dE_g/dxi = 2 b per keyframe and
  E_g = sum of the tracking energies.
* Eqs. (mean_color), (variance): E_p is quadratic in rho with curvature 2 N_j.  At
  rho* = mean colour the gradient in rho vanishes and E_p(rho* + delta) - E_p(rho*) equals
  sum_j N_j |delta_j|^2 exactly, which is the decomposition of Eq. (variance).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I


@pytest.fixture(scope="module")
def setup():
    ks = I.keyframes(seed=2, n_keyframes=4, stride=10, cam=I.TINY_160, voxel_size=0.02)
    m_ = O.OracleMap(O.params(ks.voxel_size, huber_delta=1e9))
    for i in range(len(ks.poses)):
        m_.integrate(ks.depths[i], ks.cam, ks.poses[i])
    ex = m_.extract()
    nu = O.visibility(ex["m"], ex["psi"], ex["g"], ks.voxel_size, ks.cam, ks.poses, ks.depths)
    rng = np.random.default_rng(0)
    rho = rng.uniform(0.2, 0.9, size=(len(ex["psi"]), 3))
    return ks, m_, ex, nu, rho


def _twist(xi):
    w, u = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = u
    return M


def _safe_nu(ks, ex, nu, margin=1e-2, poses=None):
    """nu without the pairs whose projection lies within `margin` px of a bilinear cell boundary."""
    vs = np.float64(np.float32(ks.voxel_size))
    gh = ex["g"] / np.linalg.norm(ex["g"], axis=1, keepdims=True)
    p = ex["m"] * vs - ex["psi"][:, None] * gh
    out = nu.copy()
    for i, T in enumerate(ks.poses if poses is None else poses):
        x = (p - T[:3, 3]) @ T[:3, :3]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = ks.cam.fx * x[:, 0] / x[:, 2] + ks.cam.cx
            v = ks.cam.fy * x[:, 1] / x[:, 2] + ks.cam.cy
        near = lambda a: np.abs(a - np.round(a)) < margin  # noqa: E731
        out[i] &= ~(near(u) | near(v))
    return out


def _safe_depths(ks, margin=1e-3, poses=None):
    """Depth images with the pixels removed whose world point lies within margin * v_s of a voxel
    boundary (half-integer multiple of v_s) on any axis."""
    vs = float(np.float32(ks.voxel_size))
    cam = ks.cam
    uu, vv = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    ray = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu, float)], -1)
    out = []
    for D, T in zip(ks.depths, ks.poses if poses is None else poses):
        P = (D[..., None] * ray) @ T[:3, :3].T + T[:3, 3]
        f = P / vs + 0.5
        near = np.any(np.abs(f - np.round(f)) < margin, axis=-1)
        out.append(np.where(near, 0.0, D).astype(np.float32))
    return out


def _generators(T):
    """d/deps of exp(eps^) T at eps = 0 for eps = (omega, upsilon): six 4 x 4 matrices."""
    G = []
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        G.append(_twist(e) @ T)
    return G


def test_visibility_selects_surface_voxels_seen_by_several_frames(setup):
    ks, _, ex, nu, _ = setup
    N = nu.sum(axis=0)
    assert (N > 0).sum() > 500
    assert (N >= 2).sum() > 200


def test_visibility_against_the_analytic_scene(setup):
    """Visibility restated from the scene geometry instead of the depth images: a voxel is visible
    in a keyframe iff it is a surface voxel, its surface point projects inside the one-pixel
    margin, and the analytic scene's first hit along the ray of the nearest pixel centre lies
    within v_s of the point's depth.  Occluded points (first hit in front) and points on the far
    side of a thin surface are therefore excluded.  Disagreements are allowed only where a value
    sits within 1e-6 of a threshold (the depth images hold FP32 copies of the ray parameters)."""
    ks, _, ex, nu, _ = setup
    vs = np.float64(np.float32(ks.voxel_size))
    gh = ex["g"] / np.linalg.norm(ex["g"], axis=1, keepdims=True)
    p = ex["m"] * vs - ex["psi"][:, None] * gh
    surf = np.all(np.abs(ex["psi"][:, None] * gh) <= 0.5 * vs, axis=1)
    cam = ks.cam
    n_vis = 0
    for i, T in enumerate(ks.poses):
        x = (p - T[:3, 3]) @ T[:3, :3]  # camera coordinates R^T (p - t)
        with np.errstate(divide="ignore", invalid="ignore"):
            u = cam.fx * x[:, 0] / x[:, 2] + cam.cx
            v = cam.fy * x[:, 1] / x[:, 2] + cam.cy
        inside = (x[:, 2] > 0) & (u >= 1) & (u <= cam.width - 2) & (v >= 1) & (v <= cam.height - 2)
        cand = np.nonzero(surf & inside)[0]
        iu, iv = np.floor(u[cand] + 0.5), np.floor(v[cand] + 0.5)
        d = np.stack([(iu - cam.cx) / cam.fx, (iv - cam.cy) / cam.fy, np.ones_like(iu)], -1)
        t_hit = ks.scene.raycast(T[:3, 3], d @ T[:3, :3].T)  # z-depth
        gap = np.abs(x[cand, 2] - t_hit)
        ok = (t_hit > 0) & (t_hit <= cam.depth_max)
        expect = np.zeros(len(p), bool)
        expect[cand] = ok & (gap <= vs)
        near_tie = np.zeros(len(p), bool)
        near_tie[cand] = (np.abs(gap - vs) < 1e-6) | (np.abs(t_hit - cam.depth_max) < 1e-6)
        for th in (u - 1, cam.width - 2 - u, v - 1, cam.height - 2 - v):
            near_tie |= np.abs(th) < 1e-9
        near_tie |= np.abs(np.abs(u - np.floor(u)) - 0.5) < 1e-9
        near_tie |= np.abs(np.abs(v - np.floor(v)) - 0.5) < 1e-9
        bad = (nu[i].astype(bool) != expect) & ~near_tie
        assert not bad.any(), (i, np.nonzero(bad)[0][:10])
        n_vis += expect.sum()
        # occlusion is exercised: candidates whose first hit lies well in front of them
        assert np.sum(ok & (x[cand, 2] - t_hit > 10 * vs)) > 0
    assert n_vis > 1000


def test_gradient_matches_finite_differences(setup):
    ks, _, ex, nu, rho = setup
    lam = 0.5
    nu = _safe_nu(ks, ex, nu)
    args = (ks.voxel_size, ks.cam, ks.poses, ks.rgbs, ks.depths, nu, lam)
    E, dpsi, dg, drho, dxi, _ = O.energy(ex["m"], ex["psi"], ex["g"], rho, *args)
    assert E[1] > 0 and E[2] > 0
    rng = np.random.default_rng(1)
    seen = np.nonzero(nu.sum(axis=0) > 0)[0]
    h = 1e-6  # the energy is O(1e4): smaller steps drown in its rounding (ulp(E) / 2h)

    def fd(field, j, k):
        vals = {"psi": ex["psi"].copy(), "g": ex["g"].copy(), "rho": rho.copy()}
        out = []
        for s in (+1, -1):
            v = {key: val.copy() for key, val in vals.items()}
            if field == "psi":
                v["psi"][j] += s * h
            else:
                v[field][j, k] += s * h
            out.append(O.energy(ex["m"], v["psi"], v["g"], v["rho"], *args, grad=False)[0])
        return (out[0] - out[1]) / (2 * h)

    noise = 4 * np.spacing(E[0]) / (2 * h)  # rounding of the two energies in the difference quotient
    for j in rng.choice(seen, 12, replace=False):
        assert fd("psi", j, 0) == pytest.approx(dpsi[j], rel=1e-5, abs=noise)
        k = int(rng.integers(3))
        assert fd("g", j, k) == pytest.approx(dg[j, k], rel=1e-5, abs=noise)
        assert fd("rho", j, k) == pytest.approx(drho[j, k], rel=1e-6, abs=noise)

    # photometric pose gradient under T <- expm(xi^) T, on pairs away from the bilinear kinks
    argsp = (ks.voxel_size, ks.cam)
    hp = 1e-8
    nu = _safe_nu(ks, ex, nu)
    E0, _, _, _, dxi_p, _ = O.energy(ex["m"], ex["psi"], ex["g"], rho, *argsp, ks.poses, ks.rgbs, ks.depths, nu, 0.0)
    for i in range(len(ks.poses)):
        for k in range(6):
            e = np.zeros(6)
            e[k] = hp
            Ep = O.energy(ex["m"], ex["psi"], ex["g"], rho, *argsp,
                          [scipy.linalg.expm(_twist(e)) @ T if q == i else T for q, T in enumerate(ks.poses)],
                          ks.rgbs, ks.depths, nu, 0.0, grad=False)[0]
            Em = O.energy(ex["m"], ex["psi"], ex["g"], rho, *argsp,
                          [scipy.linalg.expm(_twist(-e)) @ T if q == i else T for q, T in enumerate(ks.poses)],
                          ks.rgbs, ks.depths, nu, 0.0, grad=False)[0]
            assert (Ep - Em) / (2 * hp) == pytest.approx(dxi_p[i, k], rel=1e-4, abs=4 * np.spacing(E0[0]) / (2 * hp))


def test_pose_matrix_gradient_matches_finite_differences(setup):
    """dE/dT for the 12 entries of every keyframe pose, photometric and geometric terms together.

    The geometric term is evaluated at the FP32 index-path point, so the poses are first rounded to
    FP32 values and stepped by h = 2^-16: T +- h is then exact in FP32 and the rounded pose moves by
    exactly +-h.  The FP32 rounding of the points themselves leaves a noise of about 1e-7 m per
    pixel, about 2e-3 in the difference quotient."""
    ks, _, ex, nu, rho = setup
    poses = [np.float32(T).astype(np.float64) for T in ks.poses]
    nu_s = _safe_nu(ks, ex, nu, margin=2e-2, poses=poses)
    depths_s = _safe_depths(ks, margin=5e-3, poses=poses)
    lam = 0.5
    base = (ex["m"], ex["psi"], ex["g"], rho, ks.voxel_size, ks.cam)
    E0, _, _, _, _, dT = O.energy(*base, poses, ks.rgbs, depths_s, nu_s, lam)
    assert E0[1] > 0 and E0[2] > 0
    h = 2.0**-16
    for i in range(len(poses)):
        for a in range(3):
            for b in range(4):
                vals = []
                for sgn in (+1, -1):
                    Ts = [T.copy() for T in poses]
                    Ts[i][a, b] += sgn * h
                    assert np.float32(Ts[i][a, b]) == Ts[i][a, b]
                    vals.append(O.energy(*base, Ts, ks.rgbs, depths_s, nu_s, lam, grad=False)[0])
                fd = (vals[0] - vals[1]) / (2 * h)
                assert fd == pytest.approx(dT[i, a, b], rel=2e-5, abs=1e-2), (i, a, b)
        assert np.all(dT[i, 3] == 0)


def test_twist_gradient_is_matrix_gradient_on_the_generators(setup):
    ks, _, ex, nu, rho = setup
    _, _, _, _, dxi, dT = O.energy(ex["m"], ex["psi"], ex["g"], rho, ks.voxel_size, ks.cam, ks.poses, ks.rgbs,
                                   ks.depths, nu, 0.5)
    for i, T in enumerate(ks.poses):
        want = np.array([np.sum(dT[i] * Gk) for Gk in _generators(T)])
        assert np.allclose(dxi[i], want, rtol=1e-6, atol=1e-9 * np.abs(want).max())


def test_geometric_pose_gradient_equals_tracking_reduction(setup):
    ks, m_, ex, nu, rho = setup
    none = np.zeros_like(nu)
    E, _, _, _, dxi, _ = O.energy(ex["m"], ex["psi"], ex["g"], rho, ks.voxel_size, ks.cam, ks.poses, ks.rgbs,
                               ks.depths, none, 1.0)
    E_track = 0.0
    for i, T in enumerate(ks.poses):
        st = m_.track_reduce(ks.depths[i], ks.cam, T)
        assert st.n_huber == 0 and st.n_valid > 1000
        assert np.allclose(dxi[i], 2 * np.array(st.b), rtol=1e-9, atol=1e-12)
        E_track += st.energy
    assert E[2] == pytest.approx(E_track, rel=1e-12)
    assert E[1] == 0.0


def test_mean_colour_minimises_and_variance_decomposition(setup):
    ks, _, ex, nu, _ = setup
    args = (ks.voxel_size, ks.cam, ks.poses, ks.rgbs, ks.depths, nu, 0.0)
    N = nu.sum(axis=0).astype(np.float64)
    zero = np.zeros((len(N), 3))
    _, _, _, d0, _, _ = O.energy(ex["m"], ex["psi"], ex["g"], zero, *args)
    seen = N > 0
    rho_star = np.zeros_like(zero)
    rho_star[seen] = -d0[seen] / (2 * N[seen, None])  # Eq. (mean_color)
    E_star, _, _, d_star, _, _ = O.energy(ex["m"], ex["psi"], ex["g"], rho_star, *args)
    assert np.max(np.abs(d_star)) < 1e-10
    rng = np.random.default_rng(3)
    delta = rng.normal(size=zero.shape) * 0.05
    E_delta = O.energy(ex["m"], ex["psi"], ex["g"], rho_star + delta, *args, grad=False)
    assert E_delta[1] - E_star[1] == pytest.approx(np.sum(N[:, None] * delta**2), rel=1e-9)
    assert np.all(rho_star[seen] >= 0.1) and np.all(rho_star[seen] <= 1.0)  # colours of the albedo range
