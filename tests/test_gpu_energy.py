"""The voxel energy's adjoint on the GPU (gsdf_energy_*) against the FP64 oracle and finite
differences.

Inputs: RGB-D keyframes of the room scene (seeded value-noise albedo), a voxel list fused by the
oracle at the true poses, psi and g rounded to FP32 (the GPU's input type; the oracle receives
the same rounded values), random colours rho.  Two sizes: 4 keyframes of 160 x 120 at 2 cm, and
the full workload, 10 keyframes of 640 x 480 at 1 cm.

Bars:
  * visibility: bit-exact (both sides decide on the FP32 index path);
  * energies: relative 1e-5 (FP32 terms, FP64 accumulation);
  * gradients: the GPU evaluates each term in FP32.  A surface point at |p| ~ 4 m carries an
    absolute rounding of ~2.4e-7 m, ~1e-4 px after projection, so each photometric term has a
    relative error of about 1e-4 of its own size.  The per-voxel bar is
    |gpu - oracle| <= 1e-3 |oracle| + 1e-4 max|oracle| (field-wise); the pose gradients, sums
    over all points, within relative 1e-4 of their largest entry;
  * finite differences of the GPU energy (1000 random entries at full size): FP32 positions
    quantise the step (ulp(u) ~ 6e-5 px against steps of 0.01 - 0.05 px) so the bar is 2 % of the
    entry plus 1e-3 of the field's largest entry; only voxels whose projections stay 0.1 px away
    from every bilinear cell boundary are sampled, so no kink lies inside the step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


def _case(n_keyframes, cam, vs):
    ks = I.keyframes(seed=2, n_keyframes=n_keyframes, stride=10, cam=cam, voxel_size=vs)
    om = O.OracleMap(O.params(ks.voxel_size))
    for i in range(len(ks.poses)):
        om.integrate(ks.depths[i], ks.cam, ks.poses[i])
    ex = om.extract()
    psi = ex["psi"].astype(np.float32)
    g = ex["g"].astype(np.float32)
    rho = np.random.default_rng(0).uniform(0.2, 0.9, size=(len(psi), 3)).astype(np.float32)
    return ks, ex["m"].astype(np.int32), psi, g, rho


@pytest.fixture(scope="module")
def small():
    return _case(4, I.TINY_160, 0.02)


@pytest.fixture(scope="module")
def full():
    return _case(10, I.KINECT_640, 0.01)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pack(nu):
    """(F, n) 0/1 visibility -> the library's bit set: (n, ceil(F / 32)) int32, bit i % 32 of word i // 32."""
    F, n = nu.shape
    words = np.zeros((n, (F + 31) // 32), np.uint64)
    for i in range(F):
        words[:, i // 32] |= nu[i].astype(np.uint64) << np.uint64(i % 32)
    return words.astype(np.uint32).view(np.int32)


def _unpack(words, F):
    w = np.asarray(words).view(np.uint32)
    return np.stack([(w[:, i // 32] >> (i % 32)) & 1 for i in range(F)]).astype(np.uint8)


def _energy(G, ks, m, depths=None):
    return G.Energy(_dev(m), ks.voxel_size, G.intrinsics(ks.cam), _dev(ks.rgbs),
                    _dev(ks.depths if depths is None else np.stack(depths)))


def _poses(ks, poses=None):
    return _dev(np.stack(ks.poses if poses is None else poses).astype(np.float64))


def _oracle(ks, m, psi, g, rho, nu, lam, poses=None):
    return O.energy(m, psi.astype(np.float64), g.astype(np.float64), rho.astype(np.float64), ks.voxel_size, ks.cam,
                    ks.poses if poses is None else poses, ks.rgbs, ks.depths, nu, lam)


def _close(gpu, orc, rel=1e-3, floor=1e-4):
    gpu, orc = np.asarray(gpu, np.float64), np.asarray(orc, np.float64)
    err = np.abs(gpu - orc)
    bound = rel * np.abs(orc) + floor * np.abs(orc).max()
    return err.max(), bool(np.all(err <= bound))


def _check_against_oracle(G, case, lam):
    ks, m, psi, g, rho = case
    en = _energy(G, ks, m)
    P = _poses(ks)
    nu = en.visibility(_dev(psi), _dev(g), P)
    nu_o = O.visibility(m, psi.astype(np.float64), g.astype(np.float64), ks.voxel_size, ks.cam, ks.poses, ks.depths)
    assert np.array_equal(nu.cpu().numpy(), _pack(nu_o)), "visibility differs"
    E, dpsi, dg, drho, dT, dxi = en.eval(_dev(psi), _dev(g), _dev(rho), P, nu, lam)
    Eo, dpsi_o, dg_o, drho_o, dxi_o, dT_o = _oracle(ks, m, psi, g, rho, nu_o, lam)
    E = E.cpu().numpy()
    assert E[1] == pytest.approx(Eo[1], rel=1e-5) and E[2] == pytest.approx(Eo[2], rel=1e-5)
    assert E[0] == pytest.approx(Eo[0], rel=1e-5)
    for name, a, b in (("dpsi", dpsi, dpsi_o), ("dg", dg, dg_o), ("drho", drho, drho_o)):
        err, ok = _close(a.cpu().numpy(), b)
        print(f"{name}: max |gpu - oracle| = {err:.3e} (max |oracle| {np.abs(b).max():.3e})")
        assert ok, name
    for name, a, b in (("dT", dT, dT_o), ("dxi", dxi, dxi_o)):
        a = a.cpu().numpy()
        err = np.abs(a - b).max()
        print(f"{name}: max |gpu - oracle| = {err:.3e} (max |oracle| {np.abs(b).max():.3e})")
        assert err <= 1e-4 * np.abs(b).max(), name
    # the energy-only launch gives the same energies
    E2 = en.eval(_dev(psi), _dev(g), _dev(rho), P, nu, lam, grad=False).cpu().numpy()
    assert np.allclose(E2, E, rtol=1e-6)
    en.close()
    return nu_o


def test_small_case_matches_oracle(G, small):
    nu = _check_against_oracle(G, small, 0.5)
    assert nu.sum() > 1000


def test_full_keyframe_set_matches_oracle(G, full):
    nu = _check_against_oracle(G, full, 0.5)
    assert nu.sum() > 10**5


def _safe_voxels(ks, m, psi, g, nu, margin):
    """Voxels every visible projection of which stays `margin` px away from a cell boundary."""
    vs = np.float64(np.float32(ks.voxel_size))
    g64 = g.astype(np.float64)
    gh = g64 / np.linalg.norm(g64, axis=1, keepdims=True)
    p = m * vs - psi.astype(np.float64)[:, None] * gh
    ok = nu.sum(axis=0) > 0
    for i, T in enumerate(ks.poses):
        x = (p - T[:3, 3]) @ T[:3, :3]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = ks.cam.fx * x[:, 0] / x[:, 2] + ks.cam.cx
            v = ks.cam.fy * x[:, 1] / x[:, 2] + ks.cam.cy
        near = (np.abs(u - np.round(u)) < margin) | (np.abs(v - np.round(v)) < margin)
        ok &= ~(nu[i].astype(bool) & near)
    return np.nonzero(ok)[0]


def test_finite_differences_on_1000_entries(G, full):
    """Central differences of the GPU energy (energy-only launches) on 1000 random entries of psi, g
    and rho, against the GPU gradient."""
    ks, m, psi, g, rho = full
    en = _energy(G, ks, m)
    P = _poses(ks)
    psi_t, g_t, rho_t = _dev(psi), _dev(g), _dev(rho)
    nu = en.visibility(psi_t, g_t, P)
    lam = 0.5
    _, dpsi, dg, drho, _, _ = en.eval(psi_t, g_t, rho_t, P, nu, lam)
    grads = {"psi": dpsi.cpu().numpy()[:, None], "g": dg.cpu().numpy(), "rho": drho.cpu().numpy()}
    cand = _safe_voxels(ks, m, psi, g, _unpack(nu.cpu().numpy(), len(ks.poses)), 0.1)
    assert len(cand) > 5000
    rng = np.random.default_rng(7)
    host = {"psi": psi[:, None], "g": g, "rho": rho}
    dev = {"psi": psi_t.view(-1, 1), "g": g_t, "rho": rho_t}
    bad = []
    for t in range(1000):
        field = ("psi", "g", "rho")[t % 3]
        j = int(rng.choice(cand))
        k = 0 if field == "psi" else int(rng.integers(3))
        # steps: psi 2e-4 m (|du| ~ f/z * 2e-4 ~ 0.05 px); g 3e-3 |g_j| (ghat turns by <= 3e-3 rad);
        # rho 1e-2 (E is quadratic in rho)
        h = {"psi": 2e-4, "g": 3e-3 * float(np.linalg.norm(g[j])), "rho": 1e-2}[field]
        base = np.float32(host[field][j, k])
        vp, vm = np.float32(base + np.float32(h)), np.float32(base - np.float32(h))
        vals = []
        for v in (vp, vm):
            dev[field][j, k] = float(v)
            vals.append(en.eval(psi_t, g_t, rho_t, P, nu, lam, grad=False)[0].item())
        dev[field][j, k] = float(base)
        fd = (vals[0] - vals[1]) / (np.float64(vp) - np.float64(vm))
        ref = grads[field][j, k]
        if abs(fd - ref) > 2e-2 * abs(ref) + 1e-3 * np.abs(grads[field]).max():
            bad.append((field, j, k, fd, ref))
    en.close()
    assert not bad, bad[:5]


def test_pose_gradient_by_finite_differences_small(G, small):
    """dE/dT of the GPU against central differences of the GPU energy in each of the 12 entries of
    every pose.  FP32-exact poses are stepped by 2^-14 (the rounded pose then moves by exactly
    +-h); the depth images drop the pixels whose point lies within 2e-2 v_s of a voxel boundary
    and the visibility keeps the pairs 0.1 px away from the cell boundaries, so no discrete choice
    changes within the step."""
    ks, m, psi, g, rho = small
    poses = [np.float32(T).astype(np.float64) for T in ks.poses]
    vs = float(np.float32(ks.voxel_size))
    cam = ks.cam
    uu, vv = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    ray = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu, float)], -1)
    depths = []
    for D, T in zip(ks.depths, poses):
        f = ((D[..., None] * ray) @ T[:3, :3].T + T[:3, 3]) / vs + 0.5
        depths.append(np.where(np.any(np.abs(f - np.round(f)) < 2e-2, axis=-1), 0.0, D).astype(np.float32))
    en = _energy(G, ks, m, depths)
    P = _poses(ks, poses)
    nu = _unpack(en.visibility(_dev(psi), _dev(g), P).cpu().numpy(), len(poses))
    keep = _safe_voxels(ks, m, psi, g, nu, 0.1)
    mask = np.zeros(nu.shape[1], bool)
    mask[keep] = True
    nu_t = _dev(_pack(nu * mask[None, :]))
    lam = 0.5
    args = (_dev(psi), _dev(g), _dev(rho))
    _, _, _, _, dT, _ = en.eval(*args, P, nu_t, lam)
    dT = dT.cpu().numpy()
    h = 2.0**-14
    for i in range(len(poses)):
        for a in range(3):
            for b in range(4):
                vals = []
                for s in (+1, -1):
                    Ts = [T.copy() for T in poses]
                    Ts[i][a, b] += s * h
                    vals.append(en.eval(*args, _dev(np.stack(Ts)), nu_t, lam, grad=False)[0].item())
                fd = (vals[0] - vals[1]) / (2 * h)
                assert fd == pytest.approx(dT[i, a, b], rel=1e-2, abs=1e-3 * np.abs(dT[i]).max()), (i, a, b)
    en.close()


def test_autograd_function_chains_through_the_pose(G, small):
    """torch.autograd: the psi / g / rho gradients equal gsdf_energy_eval's, scaled by the incoming
    gradient, and the pose-matrix gradient chained through T(xi) = expm(xi^) T at xi = 0 gives
    the left-perturbation gradient dxi."""
    ks, m, psi, g, rho = small
    en = _energy(G, ks, m)
    P0 = _poses(ks)
    psi_t, g_t, rho_t = _dev(psi), _dev(g), _dev(rho)
    nu = en.visibility(psi_t, g_t, P0)
    lam = 0.5
    E_ref, dpsi, dg, drho, dT, dxi = en.eval(psi_t, g_t, rho_t, P0, nu, lam)
    xi = torch.zeros((len(ks.poses), 6), dtype=torch.float64, device="cuda", requires_grad=True)
    w0, w1, w2, u0, u1, u2 = xi.unbind(1)
    z = torch.zeros_like(w0)
    hat = torch.stack([torch.stack([z, -w2, w1, u0], -1), torch.stack([w2, z, -w0, u1], -1),
                       torch.stack([-w1, w0, z, u2], -1), torch.stack([z, z, z, z], -1)], -2)
    poses = torch.matrix_exp(hat) @ P0
    ps, gs, rs = (x.clone().requires_grad_(True) for x in (psi_t, g_t, rho_t))
    E = G.voxel_energy(ps, gs, rs, poses, en, nu, lam)
    assert E.item() == pytest.approx(E_ref[0].item(), rel=1e-6)  # energy-only vs gradient launch
    (3.0 * E).backward()
    # the kernels scale each contribution in FP32 and the geometric term adds with FP32 atomics in
    # no fixed order, so entries where terms cancel differ by a few roundings of the field's scale
    for got, want in ((ps.grad, dpsi), (gs.grad, dg), (rs.grad, drho)):
        assert torch.allclose(got, 3.0 * want, rtol=1e-5, atol=1e-6 * want.abs().max().item())
    # pose sums: FP32 warp partials whose grouping follows the (atomic) order of the visible-voxel list
    assert torch.allclose(xi.grad, 3.0 * dxi, rtol=1e-5, atol=1e-6 * dxi.abs().max().item())
    en.close()


def test_edge_cases(G, small):
    ks, m, psi, g, rho = small
    P = _poses(ks)
    # an empty voxel list: nothing visible, nothing hit
    en = G.Energy(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), ks.voxel_size, G.intrinsics(ks.cam),
                  _dev(ks.rgbs), _dev(ks.depths))
    empty = torch.zeros(0, device="cuda")
    E, dpsi, _, _, dT, dxi = en.eval(empty, empty, empty, P, torch.zeros((0, 1), dtype=torch.int32, device="cuda"), 0.5)
    assert E.cpu().numpy().tolist() == [0.0, 0.0, 0.0] and dpsi.numel() == 0
    assert torch.count_nonzero(dT).item() == 0 and torch.count_nonzero(dxi).item() == 0
    en.close()
    # a repeated voxel is rejected
    with pytest.raises(G.GsdfError):
        G.Energy(_dev(np.concatenate([m, m[:1]])), ks.voxel_size, G.intrinsics(ks.cam), _dev(ks.rgbs), _dev(ks.depths))
    # lambda = 0: no geometric term; nothing visible: no photometric term
    en = _energy(G, ks, m)
    psi_t, g_t, rho_t = _dev(psi), _dev(g), _dev(rho)
    nu = en.visibility(psi_t, g_t, P)
    E0 = en.eval(psi_t, g_t, rho_t, P, nu, 0.0, grad=False).cpu().numpy()
    assert E0[2] == 0.0 and E0[0] == E0[1] > 0
    none = torch.zeros_like(nu)
    E1, dpsi, dg, drho, _, _ = en.eval(psi_t, g_t, rho_t, P, none, 0.5)
    E1 = E1.cpu().numpy()
    assert E1[1] == 0.0 and E1[2] > 0 and torch.count_nonzero(drho).item() == 0
    # the geometric-only gradient against the oracle
    Eo, dpsi_o, dg_o, _, dxi_o, _ = _oracle(ks, m, psi, g, rho, np.zeros((len(ks.poses), len(m)), np.uint8), 0.5)
    assert E1[2] == pytest.approx(Eo[2], rel=1e-5)
    assert _close(dpsi.cpu().numpy(), dpsi_o)[1] and _close(dg.cpu().numpy(), dg_o)[1]
    # argument errors
    L = G.load_library()
    assert L.gsdf_energy_eval(None, None, None, None, None, None, 0.0, None, None, None, None, None, None,
                              None) == G.GSDF_ERR_INVALID_ARG
    en.close()
