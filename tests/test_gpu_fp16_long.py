"""The FP16 payload over a 300-frame sequence (the room at 4 mm voxels, 0.5 cm per frame), against
the FP64 oracle in lockstep.

The GPU runs the whole SLAM loop (10 Gauss-Newton steps then fusion per frame) with the FP16
payload.  The oracle fuses every frame at the GPU's tracked pose, so both maps see the same
decisions; at frames 1, 10, 100 and 300 it also tracks the frame from the GPU's previous pose
against its own map.  Bars at each checkpoint c:
  * pose: the oracle's 10 steps land within 1e-4 of the GPU's (the library's pose tolerance);
  * voxel set: identical (decided on the FP32 index path from the same poses);
  * psi: each frame's re-encode adds at most 2^-11 sigma_b <= 2^-11 T to a voxel, and an earlier
    error enters the next average with weight W / W' <= 1, so after c frames
    |psi - psi_oracle| <= c 2^-11 T (plus FP32 noise);
  * ghat: its mean error stays below 1e-3 (the per-frame half-precision level); the maximum is
    printed with the other figures;
  * the track is kept: the position stays within 5 cm of the truth (the sequence is drawn so that
    every view constrains all six degrees of freedom; a frame-to-model tracker without loop
    closure drifts with the path length, and a lost track jumps by tens of centimetres).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_parity import _ghat, _sorted  # noqa: E402

FRAMES = 300
CHECKS = (1, 10, 100, 300)
VOXEL = 0.004


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


@pytest.fixture(scope="module")
def seq():
    return I.room_sequence(seed=2, n_frames=FRAMES + 1, voxel_size=VOXEL, frames_per_segment=75, processes=8,
                           conditioned_horizon=FRAMES + 1)


def test_fp16_300_frames_against_oracle(G, seq):
    s = seq
    T_trunc = 5 * VOXEL
    K = G.intrinsics(s.cam)
    m = G.Map(G.make_config(VOXEL, hash_slots=1 << 17, fp16=True, max_touched_blocks=1 << 16))
    depths = torch.from_numpy(s.depths).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(s.poses[0])).cuda()
    m.integrate(depths[0], K, pose)
    track = torch.zeros((FRAMES + 1, 4, 4), dtype=torch.float64, device="cuda")
    track[0] = pose
    fields = {}
    for f in range(1, FRAMES + 1):
        m.track(depths[f], K, pose, 10)
        track[f] = pose
        m.integrate(depths[f], K, pose)
        if f in CHECKS:
            fields[f] = _sorted(m.extract())
    m.sync()
    poses = track.cpu().numpy()
    m.close()

    om = O.OracleMap(O.params(VOXEL))
    om.integrate(s.depths[0], s.cam, s.poses[0])
    for f in range(1, FRAMES + 1):
        if f in CHECKS:
            To = poses[f - 1].copy()
            for _ in range(10):
                To, _ = om.track_step(s.depths[f], s.cam, To)
            dpose = np.abs(To - poses[f]).max()
        om.integrate(s.depths[f], s.cam, poses[f])
        if f in CHECKS:
            gv, ov = fields[f], om.extract()
            assert np.array_equal(gv["m"], ov["m"]), f"voxel sets differ at frame {f}"
            dpsi = np.abs(gv["psi"] - ov["psi"])
            dg = np.abs(_ghat(gv["g"].astype(np.float64)) - _ghat(ov["g"])).max(axis=1)
            err = np.linalg.norm(poses[f][:3, 3] - s.poses[f][:3, 3])
            print(f"frame {f}: {len(gv)} voxels, pose vs oracle {dpose:.2e}, |dpsi| max {dpsi.max():.2e} "
                  f"mean {dpsi.mean():.2e} (bound {f * 2**-11 * T_trunc:.2e}), |dghat| max {dg.max():.2e} "
                  f"mean {dg.mean():.2e}, position error vs truth {err:.2e} m")
            assert dpose < 1e-4, (f, dpose)
            assert err < 0.05, (f, err)  # drifts with the path, but stays tracked
            assert dpsi.max() <= f * 2**-11 * T_trunc + 1e-6, f
            assert dg.mean() <= 1e-3, f
