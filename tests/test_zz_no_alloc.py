"""The allocation-free tracking step, called through the C ABI.

gsdf_track_step_dense_noalloc serves callers that may not allocate device memory (their device
memory is owned and handed out by a host framework, or they run in a real-time loop where an
allocation and the synchronisation it can cause are not allowed).  It must give the same result
as the handle-based gsdf_track_step on the same grid, call after call, while taking its scratch
from a static array inside the library.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_track_step_matches_handle_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf as G

    G.load_library()
    c = I.dense_sphere_case(1)
    damping = 1e-4
    K = G.intrinsics(c.cam)
    depth = torch.from_numpy(c.depth).cuda()

    # reference: the handle-based entry point on the same grid
    cfg = G.make_config(c.voxel_size, dense_dims=c.dims, dense_origin=c.origin, damping=damping)
    m = G.Map(cfg)
    m.upload_dense(c.psi, c.grad, c.weight)
    pose_ref = torch.from_numpy(np.ascontiguousarray(c.T_init)).cuda()
    stats_ref = m.new_track_stats(2)

    # the caller's own grid in the library's dense payload layout: (W psi, g) and W, x fastest
    w = c.weight.reshape(-1).astype(np.float32)
    A = np.concatenate([(w * c.psi.reshape(-1).astype(np.float32))[:, None],
                        c.grad.reshape(-1, 3).astype(np.float32)], axis=1)
    A_dev = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    W_dev = torch.from_numpy(w).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(c.T_init)).cuda()
    stats = torch.zeros((2, G.TRACK_STATS_BYTES), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    for call in range(2):
        m.track_step(depth, K, pose_ref, stats_ref[call])
        st = G.gsdf_track_step_dense_noalloc(depth.data_ptr(), K, A_dev.data_ptr(), W_dev.data_ptr(), c.dims,
                                             c.origin, c.voxel_size, c.voxel_size, damping, pose.data_ptr(),
                                             stats[call].data_ptr(), stream)
        assert st == G.GSDF_OK, G.gsdf_status_string(st)
        torch.cuda.synchronize()
        a = G.track_stats_from_bytes(stats_ref[call].cpu().numpy())
        b = G.track_stats_from_bytes(stats[call].cpu().numpy())
        assert a.status == b.status == G.GSDF_OK
        assert a.n_valid == b.n_valid > 5000
        # the same kernel with the same grid over the same inputs, and grid sums that are exact in
        # any order: the statistics (H, b, energy, counts, increment) and the pose agree bit for bit
        assert bytes(stats_ref[call].cpu().numpy()) == bytes(stats[call].cpu().numpy()), call
        assert np.array_equal(pose.cpu().numpy(), pose_ref.cpu().numpy()), call
    m.sync()

    # invalid arguments are rejected before anything is launched
    bad = G.gsdf_track_step_dense_noalloc(depth.data_ptr(), K, A_dev.data_ptr(), W_dev.data_ptr(), (0, 64, 64),
                                          c.origin, c.voxel_size, c.voxel_size, damping, pose.data_ptr())
    assert bad == G.GSDF_ERR_INVALID_ARG
