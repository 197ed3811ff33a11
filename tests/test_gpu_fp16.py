"""FP16 voxel payload with per-block scale, against the FP64 oracle.

The FP16 form stores psi / sigma_b and gbar = g / W in half precision (sigma_b = the largest |psi|
its block has held, at most T) and W in FP32; per-pixel arithmetic stays FP32.  The discrete
decisions (voxel set, block set) do not involve the payload and must match the oracle bit for
bit.  The values carry the rounding of half precision (unit roundoff 2^-11):
  * psi: each frame re-encodes a touched voxel once, and a decoded value enters the next average
    with weight W / W' < 1, so |psi - psi_oracle| <= 2 * 2^-11 * T plus FP32 noise;
  * ghat: gbar components round with relative error 2^-11, so |ghat - ghat_oracle| <= 1e-3;
  * W: FP32, as in the FP32 form (1e-5 relative).
The pose gate stays 1e-4 (rad / m) after 10 Gauss-Newton steps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_parity import _ghat, _sorted  # noqa: E402


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


@pytest.fixture(scope="module")
def room4mm():
    return I.room_sequence(seed=2, n_frames=4, voxel_size=0.004)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _fp16_map(G, vs, slots=1 << 17, cap=None):
    return G.Map(G.make_config(vs, hash_slots=slots, fp16=True, max_touched_blocks=cap or slots // 2))


def test_fp16_fusion_matches_oracle_within_half_precision(G, room4mm):
    s = room4mm
    T = 5 * s.voxel_size
    m = _fp16_map(G, s.voxel_size)
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    st = m.new_integrate_stats()
    for f in range(2):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]), st)
        ost = om.integrate(s.depths[f], s.cam, s.poses[f])
        g = G.integrate_stats_from_bytes(st.cpu().numpy())
        assert g.n_rays == ost.n_rays and g.n_visits == ost.n_visits
    m.sync()
    gv, ov = _sorted(m.extract()), om.extract()
    assert len(gv) > 10**6
    assert np.array_equal(gv["m"], ov["m"]), "voxel sets differ"
    dpsi = np.abs(gv["psi"] - ov["psi"])
    dg = np.abs(_ghat(gv["g"].astype(np.float64)) - _ghat(ov["g"]))
    print(f"fp16 payload: max |dpsi| = {dpsi.max():.3e} (bound {2 * 2**-11 * T:.3e}), max |dghat| = {dg.max():.3e}")
    assert dpsi.max() <= 2 * 2**-11 * T + 1e-6
    assert dg.max() <= 1e-3
    assert np.max(np.abs(gv["w"] - ov["w"]) / ov["w"]) <= 1e-5


def test_fp16_tracking_pose_matches_oracle(G, room4mm):
    s = room4mm
    m = _fp16_map(G, s.voxel_size)
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    for f in range(2):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
        om.integrate(s.depths[f], s.cam, s.poses[f])
    pose = _dev(s.poses[1])
    T = s.poses[1].copy()
    d = _dev(s.depths[2])
    m.track(d, K, pose, 10)
    for _ in range(10):
        T, _ = om.track_step(s.depths[2], s.cam, T)
    m.sync()
    diff = np.abs(pose.cpu().numpy() - T).max()
    print(f"fp16 payload: pose difference after 10 steps {diff:.3e}")
    assert diff < 1e-4


def test_fp16_checkpoint_roundtrip_and_capacity(G, room4mm):
    s = room4mm
    T = 5 * s.voxel_size
    m = _fp16_map(G, s.voxel_size)
    K = G.intrinsics(s.cam)
    m.integrate(_dev(s.depths[0]), K, _dev(s.poses[0]))
    a = m.extract()
    m2 = _fp16_map(G, s.voxel_size)
    m2.load(a)
    b = m2.extract()
    assert np.array_equal(a["m"], b["m"]) and np.array_equal(a["w"], b["w"])
    assert np.max(np.abs(a["psi"] - b["psi"])) <= 2**-11 * T + 1e-7
    # a per-frame accumulator far too small: partial fusion, reported as capacity
    small = _fp16_map(G, s.voxel_size, cap=16)
    small.integrate(_dev(s.depths[0]), K, _dev(s.poses[0]))
    assert G.gsdf_sync(small.h) == G.GSDF_ERR_CAPACITY
    assert 0 < small.num_blocks()
    with pytest.raises(G.GsdfError):
        G.Batch([m])  # FP16 handles are not batched
