"""The allocation-free entry point, kkm_distances_noalloc.

Some callers cannot allocate device memory: a process whose memory a caching
allocator or a pre-sized arena owns, or a loop where cudaMalloc's device
synchronisation is not acceptable. kkm_distances_noalloc lets them score query
points against centers they hold themselves. Its only scratch is a fixed
array inside the library.

Through the C ABI, this file checks that:
- the call gives the distances of Eq. (1)'s weighted centers that the FP64
  oracle computes directly, and the same distances and nearest centers as the
  context-based kkm_assign, for the Gaussian, Laplacian and polynomial
  kernels, with query and support rows read through strided views;
- it does so on two calls in a row, so nothing carried over in the shared
  scratch changes the second answer, and that after a first call with m = 0
  neither call changes the device's free memory;
- a center with no support row scores K(q, q) + ||C_j||^2 = K(q, q), offsets
  that are not non-decreasing give NaN distances and assignments of -1, and a
  well-formed call after them is right again;
- sizes beyond the scratch are rejected on the host.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_2410_05902_gb300 import inputs
from paper_2410_05902_gb300 import kkm as kb

KIND = {"gaussian": oracle.GAUSSIAN, "laplacian": oracle.LAPLACIAN, "poly": oracle.POLY}
DIST_TOL = 1e-5          # normwise, FP32 arithmetic against FP64 (as for the FP32 form's distance pass)
N, D, K, B = 3000, 24, 8, 256


def _params(kind, X):
    sigma = inputs.median_sigma(X, seed=1)
    if kind == "gaussian":
        return 2 * sigma * sigma, 0.0, 2
    if kind == "laplacian":
        return sigma, 0.0, 2
    return 1.0, 1.0, 2          # (<x, y> + 1)^2


def _call(Q, Y, S, w, seg, cn, k, kern, dist, assign):
    import torch
    kb.kkm_distances_noalloc(Q.data_ptr(), Q.shape[0], Q.stride(0), Q.shape[1], Y.data_ptr(), S, Y.stride(0),
                             w.data_ptr(), seg.data_ptr(), cn.data_ptr(), k, kern, dist.data_ptr(),
                             assign.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _strided(torch, A, pad, shift):
    """A device copy of A read through a view with leading dimension A.shape[1] + pad."""
    big = torch.zeros((A.shape[0], A.shape[1] + pad), dtype=torch.float32, device="cuda")
    view = big[:, shift:shift + A.shape[1]]
    view.copy_(torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)))
    assert view.stride(0) == A.shape[1] + pad
    return view


def _warm_up(torch):
    # the first call on the device, with m = 0, loads the scratch and the kernels
    kb.kkm_distances_noalloc(0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, None, None, None,
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def _fitted(kind):
    import torch
    from paper_2410_05902_gb300.kkm import KKM
    X, _ = inputs.isotropic_mixture(N, D, K, seed=77)
    X = X.astype(np.float32)
    param, coef0, degree = _params(kind, X)
    run = KKM(torch.from_numpy(X).cuda(), K, B, kernel=kind, param=param, coef0=coef0, degree=degree, tau=150,
              precision="fp32", init_idx=inputs.init_indices(len(X), K, seed=5))
    for batch in inputs.batch_stream(len(X), B, 6, seed=8):
        run.step(torch.from_numpy(batch.astype(np.int32)).cuda())
    st = run.get_state()
    kern = kb.kkm_kernel(kb.KERNELS[kind], float(param), float(coef0), int(degree))
    okern = oracle.Kernel(KIND[kind], float(param), float(coef0), int(degree))
    # query points: 1500 data rows plus 700 fresh points (m > one pass of 1024 rows)
    fresh, _ = inputs.isotropic_mixture(700, D, K, seed=78)
    Q = np.ascontiguousarray(np.concatenate([X[:1500], fresh.astype(np.float32)]))
    return run, X, st, kern, okern, Q


def _held(torch, X, st):
    """The centers as a caller holds them: strided support rows, weights, offsets, norms."""
    Y = _strided(torch, X[st["row_idx"]], 5, 1)
    w = torch.from_numpy(np.asarray(st["row_w"], np.float32)).cuda()
    seg = torch.from_numpy(np.concatenate([[0], np.cumsum(st["rows_per_center"])]).astype(np.int32)).cuda()
    cn = torch.from_numpy(np.asarray(st["cnorm"], np.float64)).cuda()
    return Y, w, seg, cn, int(np.sum(st["rows_per_center"]))


# Both calls accumulate the Laplacian kernel's ||q - y||^2 from differences
# (through ||q||^2 + ||y||^2 - 2 <q, y> a query equal to a support row would
# keep d2 ~ eps ||q||^2, which the square root magnifies), so every kernel is
# held to the FP32 bound against kkm_assign too.
ASSIGN_TOL = {"gaussian": DIST_TOL, "laplacian": DIST_TOL, "poly": DIST_TOL}


def _check(d, a, d_ref, what, tol=DIST_TOL):
    scale = float(np.max(np.abs(d_ref)))
    err = float(np.max(np.abs(d - d_ref))) / scale
    assert err <= tol, f"{what}: normwise distance difference {err:.3e}"
    order = np.sort(d_ref, axis=1)
    bad = np.nonzero(a != np.argmin(d_ref, axis=1))[0]
    assert np.all(order[bad, 1] - order[bad, 0] <= 2 * tol * scale), f"{what}: assignments differ"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # argument checks come before any CUDA call, so this runs without a GPU
    lib = kb.load()
    with pytest.raises(kb.KKMError, match="KKM_NOALLOC_MAX_SUPPORT"):
        kb.kkm_distances_noalloc(0x1000, 10, 8, 8, 0x1000, 65537, 8, 0x1000, 0x1000, 0x1000, 4,
                                 kb.kkm_kernel(kb.KKM_GAUSSIAN, 1.0, 0.0, 2), None, None, None)
    with pytest.raises(kb.KKMError, match="KKM_NOALLOC_MAX_TILES"):
        kb.kkm_distances_noalloc(0x1000, 10, 8, 8, 0x1000, 60000, 8, 0x1000, 0x1000, 0x1000, 200,
                                 kb.kkm_kernel(kb.KKM_GAUSSIAN, 1.0, 0.0, 2), None, None, None)
    with pytest.raises(kb.KKMError, match="m must be >= 0"):
        kb.kkm_distances_noalloc(0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, None, None, None, None)
    assert lib.kkm_noalloc_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["gaussian", "laplacian", "poly"])
def test_noalloc_matches_oracle_and_kkm_assign_on_two_calls(kind):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _warm_up(torch)
    run, X, st, kern, okern, Qh = _fitted(kind)
    Y, w, seg, cn, S = _held(torch, X, st)
    Q = _strided(torch, Qh, 8, 3)
    m = Qh.shape[0]
    a_ref, _, d_ref = run.assign(torch.from_numpy(Qh).cuda(), want_dist=True)
    torch.cuda.synchronize()
    d_ref = d_ref.cpu().numpy().astype(np.float64)
    del a_ref   # the assignments are checked against argmin of the distances, up to near ties
    d_ora, _ = oracle.state_distances(X.astype(np.float64), Qh.astype(np.float64), st, okern)
    outs = [(torch.full((m, K), float("nan"), dtype=torch.float32, device="cuda"),
             torch.full((m,), -1, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    for call, (dist, assign) in enumerate(outs):
        free0 = torch.cuda.mem_get_info()[0]
        _call(Q, Y, S, w, seg, cn, K, kern, dist, assign)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, f"call {call}: free device memory changed by {free0 - free1} bytes"
        d = dist.cpu().numpy().astype(np.float64)
        a = assign.cpu().numpy()
        _check(d, a, d_ora, f"{kind} call {call} vs oracle")
        _check(d, a, d_ref, f"{kind} call {call} vs kkm_assign", ASSIGN_TOL[kind])
    run.close()


@pytest.mark.gpu
def test_noalloc_empty_center_and_rejected_offsets():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _warm_up(torch)
    run, X, st, kern, okern, Qh = _fitted("gaussian")
    run.close()
    # center 3 loses its support rows: an empty segment between two full ones
    rows = np.asarray(st["rows_per_center"], np.int64)
    off = np.concatenate([[0], np.cumsum(rows)])
    keep = np.concatenate([np.arange(off[j], off[j + 1]) for j in range(K) if j != 3])
    rows_e = rows.copy()
    rows_e[3] = 0
    st_e = {"row_idx": np.asarray(st["row_idx"])[keep], "row_w": np.asarray(st["row_w"])[keep],
            "rows_per_center": rows_e}
    d_ora, cn_ora = oracle.state_distances(X.astype(np.float64), Qh.astype(np.float64), st_e, okern)
    assert cn_ora[3] == 0.0
    st_e["cnorm"] = cn_ora
    Y, w, seg, cn, S = _held(torch, X, st_e)
    Q = _strided(torch, Qh, 8, 3)
    m = Qh.shape[0]
    dist = torch.empty((m, K), dtype=torch.float32, device="cuda")
    assign = torch.empty((m,), dtype=torch.int32, device="cuda")
    _call(Q, Y, S, w, seg, cn, K, kern, dist, assign)
    torch.cuda.synchronize()
    d = dist.cpu().numpy().astype(np.float64)
    _check(d, assign.cpu().numpy(), d_ora, "empty center")
    np.testing.assert_allclose(d[:, 3], 1.0, rtol=0, atol=1e-6)      # K(q, q) = 1 for the Gaussian kernel
    # offsets that decrease (center 1's end before its start) are rejected on the device
    bad = seg.clone()
    bad[2] = bad[1] - 1
    _call(Q, Y, S, w, bad, cn, K, kern, dist, assign)
    torch.cuda.synchronize()
    assert torch.isnan(dist).all().item()
    assert (assign == -1).all().item()
    # and the next well-formed call is right again
    _call(Q, Y, S, w, seg, cn, K, kern, dist, assign)
    torch.cuda.synchronize()
    _check(dist.cpu().numpy().astype(np.float64), assign.cpu().numpy(), d_ora, "after rejected offsets")
