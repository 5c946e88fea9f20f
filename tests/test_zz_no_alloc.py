"""The allocation-free warp J^T J p entry point against the planned one.

opt_warp_apply_jtj_noalloc serves callers that cannot allocate device memory
(fixed-budget interactive loops, hosts that own all device memory); its only
scratch is a static device array.  Two calls in a row, through the C ABI, must
give the same q = J^T J p and p.q as opt_apply_jtj, within the 1e-5 relative
tolerance of the other product tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1604_06525_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_noalloc_apply_matches_planned_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1604_06525_gb300 import build, api
    build.build()
    lib = api.load_library()

    W, H = 100, 70
    prob = synth.warp_problem(W, H, 12, seed=5, mask=synth.random_mask(W, H, 0.1, 6), x0_noise=0.4)
    planned = api.Problem(prob)
    dev = torch.device("cuda")
    x = torch.as_tensor(prob.x0, device=dev).contiguous()
    U = torch.as_tensor(prob.urshape, device=dev).contiguous()
    mask = torch.as_tensor(prob.mask, dtype=torch.uint8, device=dev)
    hidx = torch.as_tensor(prob.handle_idx, dtype=torch.int32, device=dev)
    q = torch.empty(3 * W * H, dtype=torch.float32, device=dev)
    pq = torch.zeros(1, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(17)
    for call in range(2):
        p = torch.as_tensor(rng.standard_normal(3 * W * H).astype(np.float32), device=dev)
        q_ref, pq_ref = planned.apply_jtj(p)
        q.fill_(float("nan"))
        st = lib.opt_warp_apply_jtj_noalloc(W, H, x.data_ptr(), U.data_ptr(), mask.data_ptr(),
                                            hidx.data_ptr(), int(hidx.numel()), prob.w_reg, prob.w_fit,
                                            p.data_ptr(), q.data_ptr(), pq.data_ptr(), None)
        assert st == 0, api.STATUS.get(st, st)
        torch.cuda.synchronize()
        assert _rel(q.cpu().numpy(), q_ref.cpu().numpy()) <= TOL, call
        assert abs(pq.item() - pq_ref) <= TOL * abs(pq_ref), call
    planned.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1604_06525_gb300 import build, api
    build.build()
    lib = api.load_library()
    # 2049 x 2048 needs 65 * 256 = 16,640 tiles > 16,384: rejected before any device work
    st = lib.opt_warp_apply_jtj_noalloc(2049, 2048, 1, 1, None, None, 0, 1.0, 100.0, 1, 1, None, None)
    assert st == 1
    st = lib.opt_warp_apply_jtj_noalloc(0, 10, 1, 1, None, None, 0, 1.0, 100.0, 1, 1, None, None)
    assert st == 1


def test_noalloc_repeated_handles_count_per_entry():
    """Repeated handle indices (which the planned entry point rejects) each
    add their own fit residual, as the float64 oracle does with one fit row
    per handle entry."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import oracle
    from paper_1604_06525_gb300 import build, api
    build.build()
    lib = api.load_library()
    W, H = 45, 19
    prob = synth.warp_problem(W, H, 5, seed=8, x0_noise=0.3)
    prob.handle_idx = np.concatenate([prob.handle_idx, prob.handle_idx[:2], prob.handle_idx[:1]]).astype(np.int32)
    prob.handle_target = np.concatenate([prob.handle_target, prob.handle_target[:2],
                                         prob.handle_target[:1]]).astype(np.float32)
    e = oracle.make_energy(prob)
    x64 = prob.x0.reshape(-1).astype(np.float64)
    dev = torch.device("cuda")
    x = torch.as_tensor(prob.x0, device=dev).contiguous()
    U = torch.as_tensor(prob.urshape, device=dev).contiguous()
    hidx = torch.as_tensor(prob.handle_idx, dtype=torch.int32, device=dev)
    p_np = np.random.default_rng(3).standard_normal(3 * W * H).astype(np.float32)
    p = torch.as_tensor(p_np, device=dev)
    q = torch.empty(3 * W * H, dtype=torch.float32, device=dev)
    st = lib.opt_warp_apply_jtj_noalloc(W, H, x.data_ptr(), U.data_ptr(), None, hidx.data_ptr(),
                                        int(hidx.numel()), prob.w_reg, prob.w_fit, p.data_ptr(), q.data_ptr(),
                                        None, None)
    assert st == 0, api.STATUS.get(st, st)
    torch.cuda.synchronize()
    qref = oracle.apply_jtj(e, x64, p_np.astype(np.float64))
    assert _rel(q.cpu().numpy(), qref) <= TOL
