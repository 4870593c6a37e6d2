"""The allocation-free entry point against the allocating one (needs a GPU).

pd_knn_cost_static serves callers that cannot allocate device memory when they
call the library (a fixed memory budget after start-up, or a host allocator
they must not touch).  It must return what pd_build_grid + pd_knn_cost return,
call after call, although every call reuses the same fixed device array.
"""
import ctypes

import numpy as np
import pytest

from paper_2311_17604_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _d2(xyz, knn):
    x = xyz.astype(np.int64)
    out = np.full(knn.shape, -1, dtype=np.int64)
    ok = knn >= 0
    r = np.nonzero(ok)
    diff = x[knn[r]] - x[r[0]]
    out[r] = (diff * diff).sum(axis=1)
    return out


def test_static_entry_point_matches_pd_knn_cost_on_consecutive_calls():
    from paper_2311_17604_gb300 import build
    build.build()
    import paper_2311_17604_gb300.pd as pd

    L = pd.lib()
    ctx = pd.Context()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    clouds = [synth.room_scan(seed=2, n_az=240, n_el=60).xyz,       # 14,400 points
              synth.random_cloud(3, 5000, 40),                       # duplicates and ties
              synth.random_cloud(4, pd.PD_STATIC_MAX_POINTS, 3000)]  # the largest size
    for ci, x in enumerate(clouds):
        n = x.shape[0]
        xd = torch.from_numpy(x).cuda()
        # k = 16 (17 stored neighbours) is the largest user of the array:
        # run it at the largest size
        for k in ((1, 4, 16) if ci == len(clouds) - 1 else (1, 4)):
            g = pd.Grid(ctx, xd)
            cost_ref, knn_ref = pd.pd_knn_cost(g, k=k)
            g.free()
            cost_ref = cost_ref.cpu().numpy()
            d2_ref = _d2(x, knn_ref.cpu().numpy())
            for _ in range(2):  # consecutive calls share the same scratch array
                cost = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
                knn = torch.full((n, k), -7, dtype=torch.int32, device="cuda")
                rc = L.pd_knn_cost_static(_p(xd), n, k, _p(cost), _p(knn), stream)
                assert rc == pd.PD_OK
                # density costs are exact: bit-identical doubles
                assert np.array_equal(cost.cpu().numpy().view(np.int64), cost_ref.view(np.int64))
                assert np.array_equal(_d2(x, knn.cpu().numpy()), d2_ref)
    ctx.close()


def test_static_entry_point_rejects_oversized_clouds():
    import paper_2311_17604_gb300.pd as pd
    L = pd.lib()
    n = pd.PD_STATIC_MAX_POINTS + 1
    big = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.pd_knn_cost_static(_p(big), n, 1, None, None, stream) == pd.PD_ERANGE
    assert L.pd_knn_cost_static(_p(big), 10, 0, None, None, stream) == pd.PD_EINVAL
    assert L.pd_knn_cost_static(_p(big), 10, 17, None, None, stream) == pd.PD_EINVAL
    # a coordinate spread of 2^25 mm: squared distances would leave the exact range
    wide = torch.tensor([[0, 0, 0], [1 << 25, 0, 0], [5, 5, 5]], dtype=torch.int32,
                        device="cuda")
    assert L.pd_knn_cost_static(_p(wide), 3, 1, None, None, stream) == pd.PD_ERANGE
    # just inside the limit the call succeeds
    wide[1, 0] = (1 << 25) - 1
    cost = torch.empty(3, dtype=torch.float64, device="cuda")
    assert L.pd_knn_cost_static(_p(wide), 3, 1, _p(cost), None, stream) == pd.PD_OK
    torch.cuda.synchronize()
    assert cost[2].item() == 1.0 / 75.0
