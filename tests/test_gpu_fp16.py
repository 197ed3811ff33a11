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
    tri = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 10, tracker=G.GSDF_TRACKER_TRILINEAR))
    with pytest.raises(G.GsdfError):
        G.Batch([m, tri])  # the trilinear tracker is not batched


def test_fp16_in_a_batch_matches_oracle(G, room4mm):
    """An FP16 scene and an FP32 scene of the 4 mm room in one batch: three frames through
    gsdf_batch_frame (frame 0 fused at its true pose, frames 1 and 2 each fused after 10 batched
    Gauss-Newton steps), the depth pointers advanced on the device.  Each scene against the FP64
    oracle run in lockstep (the oracle
    starts every tracking run from the batch's pose and fuses at the batch's tracked pose): voxel
    set exact, psi within 2 * 2^-11 T (FP16) or 1e-5 (FP32), ghat within 1e-3 (FP16) or 1e-5,
    poses within 1e-4."""
    s = room4mm
    T = 5 * s.voxel_size
    maps = [_fp16_map(G, s.voxel_size), G.Map(G.make_config(s.voxel_size, hash_slots=1 << 17))]
    batch = G.Batch(maps)
    K = G.intrinsics(s.cam)
    depths = _dev(s.depths)
    poses = [_dev(s.poses[0]) for _ in maps]
    batch.set_frames([depths[0], depths[0]], [K, K], poses)
    batch.set_depth_stride([s.cam.width * s.cam.height] * 2)
    oms = [O.OracleMap(O.params(s.voxel_size)) for _ in maps]
    Tprev = [s.poses[0]] * 2
    for f in range(3):
        batch.frame(0 if f == 0 else 10)  # tracks frame f (f > 0), fuses it, advances to f + 1
        torch.cuda.synchronize()
        for k, om in enumerate(oms):
            Tg = poses[k].cpu().numpy()
            if f > 0:
                To = Tprev[k].copy()
                for _ in range(10):
                    To, _ = om.track_step(s.depths[f], s.cam, To)
                diff = np.abs(Tg - To).max()
                print(f"batched {'fp16' if k == 0 else 'fp32'} frame {f}: pose difference {diff:.3e}")
                assert diff < 1e-4, (k, f, diff)
            om.integrate(s.depths[f], s.cam, Tg)
            Tprev[k] = Tg
    for k, (m, om) in enumerate(zip(maps, oms)):
        m.sync()
        gv, ov = _sorted(m.extract()), om.extract()
        assert np.array_equal(gv["m"], ov["m"]), k
        dpsi = np.abs(gv["psi"] - ov["psi"]).max()
        dg = np.abs(_ghat(gv["g"].astype(np.float64)) - _ghat(ov["g"])).max()
        print(f"batched {'fp16' if k == 0 else 'fp32'}: max |dpsi| {dpsi:.3e}, max |dghat| {dg:.3e}")
        assert dpsi <= (2 * 2**-11 * T + 1e-6 if k == 0 else 1e-5)
        assert dg <= (1e-3 if k == 0 else 1e-5)
        assert np.max(np.abs(gv["w"] - ov["w"]) / ov["w"]) <= 1e-5
    batch.close()
