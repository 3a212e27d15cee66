"""The allocation-free entry point, kkm_distances_noalloc.

Some callers cannot allocate device memory: a process whose memory a caching
allocator or a pre-sized arena owns, or a loop where cudaMalloc's device
synchronisation is not acceptable. kkm_distances_noalloc lets them score query
points against centers they hold themselves. Its only scratch is a fixed
array inside the library. This file checks, through the C ABI, that it gives
the same distances and nearest centers as the context-based kkm_assign on the
same centers, on two calls in a row, so nothing carried over in the shared
scratch can change the second answer. It also checks that it rejects sizes
beyond its scratch on the host. This file is named so that pytest collects it
last.
"""
import numpy as np
import pytest

from paper_2410_05902_gb300 import inputs
from paper_2410_05902_gb300 import kkm as kb


def _kernel(kappa):
    return kb.kkm_kernel(kb.KKM_GAUSSIAN, float(kappa), 0.0, 2)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # argument checks come before any CUDA call, so this runs without a GPU
    lib = kb.load()
    too_many_rows = kb.KKMError
    with pytest.raises(too_many_rows, match="KKM_NOALLOC_MAX_SUPPORT"):
        kb.kkm_distances_noalloc(0x1000, 10, 8, 8, 0x1000, 65537, 8, 0x1000, 0x1000, 0x1000, 4,
                                 _kernel(1.0), None, None, None)
    with pytest.raises(kb.KKMError, match="KKM_NOALLOC_MAX_TILES"):
        kb.kkm_distances_noalloc(0x1000, 10, 8, 8, 0x1000, 60000, 8, 0x1000, 0x1000, 0x1000, 200,
                                 _kernel(1.0), None, None, None)
    assert lib.kkm_noalloc_last_error()


@pytest.mark.gpu
def test_noalloc_matches_kkm_assign_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05902_gb300.kkm import KKM
    X, _ = inputs.isotropic_mixture(3000, 24, 8, seed=77)
    sigma = inputs.median_sigma(X, seed=1)
    kappa = 2 * sigma * sigma
    k, b = 8, 256
    Xd = torch.from_numpy(X).cuda()
    run = KKM(Xd, k, b, kernel="gaussian", param=kappa, tau=150, precision="fp32",
              init_idx=inputs.init_indices(len(X), k, seed=5))
    for B in inputs.batch_stream(len(X), b, 6, seed=8):
        run.step(torch.from_numpy(B.astype(np.int32)).cuda())
    st = run.get_state()
    # the centers as the caller would hold them: support rows, weights, offsets, norms
    Y = torch.from_numpy(np.ascontiguousarray(X[st["row_idx"]])).cuda()
    w = torch.from_numpy(st["row_w"].astype(np.float32)).cuda()
    seg = torch.from_numpy(np.concatenate([[0], np.cumsum(st["rows_per_center"])]).astype(np.int32)).cuda()
    cn = torch.from_numpy(st["cnorm"]).cuda()
    S = int(st["rows_per_center"].sum())
    # query points: a copy of 1500 data rows plus 700 fresh points (m > one pass of 1024 rows)
    fresh, _ = inputs.isotropic_mixture(700, 24, 8, seed=78)
    Q = torch.from_numpy(np.ascontiguousarray(np.concatenate([X[:1500], fresh]))).cuda()
    m = Q.shape[0]
    a_ref, _, d_ref = run.assign(Q, want_dist=True)
    torch.cuda.synchronize()
    d_ref = d_ref.cpu().numpy().astype(np.float64)
    a_ref = a_ref.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    scale = float(np.max(np.abs(d_ref)))
    order = np.sort(d_ref, axis=1)
    for call in range(2):
        dist = torch.full((m, k), float("nan"), dtype=torch.float32, device="cuda")
        assign = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        kb.kkm_distances_noalloc(Q.data_ptr(), m, Q.stride(0), X.shape[1], Y.data_ptr(), S, Y.stride(0),
                                 w.data_ptr(), seg.data_ptr(), cn.data_ptr(), k, _kernel(kappa),
                                 dist.data_ptr(), assign.data_ptr(), stream)
        torch.cuda.synchronize()
        d = dist.cpu().numpy().astype(np.float64)
        a = assign.cpu().numpy()
        err = float(np.max(np.abs(d - d_ref))) / scale
        assert err <= 1e-5, f"call {call}: normwise distance difference {err:.3e}"
        bad = np.nonzero(a != a_ref)[0]
        assert np.all(order[bad, 1] - order[bad, 0] <= 1e-5 * scale), f"call {call}: assignments differ"
    run.close()
