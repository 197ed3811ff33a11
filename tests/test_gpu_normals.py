"""The 75 degree normal test (Sec. 5.3) near its threshold.

Fusion keeps a pixel when the angle between its normal and its viewing ray is below 75 degrees.
The kernel decides most pixels from a cheap evaluation of the cosine and falls back to the
specified correctly rounded evaluation near the threshold, so its decisions must equal the
oracle's bit for bit.  This test puts a large share of the image near the threshold: a plane at
exactly 75 degrees to the central ray, seen through a very narrow field of view (f = 2e4 px), so
the cosine varies by about 1e-3 over the image, and the central-difference normals of the FP32 depth
scatter it further.  The kept rays and the fused voxel set must match the oracle exactly, the
fused values within the parity tolerances.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_parity import _sorted  # noqa: E402


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


def _plane_depth(cam, normal, dist):
    """z-depth of the plane {x : normal . x = dist} seen from the origin along +z (FP64)."""
    d = cam.ray_dirs_cam()
    t = dist / (d @ normal)
    t = np.where(t > 0, t, 0.0)
    return t.reshape(cam.height, cam.width).astype(np.float32)


@pytest.mark.parametrize("angle_deg", [75.0, 74.99, 75.01])
def test_threshold_decisions_match_oracle(G, angle_deg):
    cam = I.Camera(2.0e4, 2.0e4, 319.5, 239.5, 640, 480, 3.5)
    a = math.radians(angle_deg)
    normal = np.array([math.sin(a), 0.0, math.cos(a)])
    depth = _plane_depth(cam, normal, 2.0 * math.cos(a))  # the central ray meets the plane at z = 2 m
    T = np.eye(4)
    vs = 5e-4  # a pixel spans 0.1 mm at 2 m: about 25 rays per voxel column, as in ordinary views
    m = G.Map(G.make_config(vs, hash_slots=1 << 14))
    st = m.new_integrate_stats()
    m.integrate(torch.from_numpy(depth).cuda(), G.intrinsics(cam), torch.from_numpy(T).cuda(), st)
    om = O.OracleMap(O.params(vs))
    ost = om.integrate(depth, cam, T)
    g = G.integrate_stats_from_bytes(st.cpu().numpy())
    n_px = cam.width * cam.height
    print(f"{angle_deg} deg: {g.n_rays} of {n_px} rays kept (oracle {ost.n_rays})")
    assert g.n_rays == ost.n_rays and g.n_visits == ost.n_visits
    if angle_deg == 75.0:
        assert 0.05 * n_px < g.n_rays < 0.95 * n_px  # the threshold splits the image
    if ost.n_rays:
        gv, ov = _sorted(m.extract()), om.extract()
        assert np.array_equal(gv["m"], ov["m"]), "voxel sets differ"
        assert np.max(np.abs(gv["psi"] - ov["psi"])) <= 1e-5
        assert np.max(np.abs(gv["w"] - ov["w"]) / ov["w"]) <= 1e-5
        # the normals of this view are very noisy (neighbouring depths differ by 1e-4 of their value
        # in FP32), so a voxel's normal sum g can nearly cancel and ghat = g / |g| would magnify
        # the last bits of each normal; the mean normal g / W has no such amplification: each unit
        # normal is within a few ulps of the oracle's, and the FP32 sum of k weighted normals adds
        # at most (k - 1) 2^-24 relative to W (4e-6 covers k <= 60 rays per voxel)
        assert np.max(np.abs(gv["g"] / gv["w"][:, None] - ov["g"] / ov["w"][:, None])) <= 4e-6
    m.sync()
    m.close()
