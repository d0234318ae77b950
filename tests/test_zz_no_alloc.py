"""The allocation-free loss entry point gives the same result as the regular one.

s3gs_mapping_loss_noalloc serves callers that cannot allocate device memory
(code inside a global-mode CUDA graph capture, hosts whose device memory is
owned by a pooling allocator or a fixed budget, loops that must not take the
implicit synchronisation of cudaMalloc/cudaFree). Its partial sums live in a
fixed static device array shared by every call, so this test calls it twice in
a row, with different inputs, and compares each result with the allocating
s3gs_mapping_loss on the same inputs. This file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_REL = 1e-5  # the same kernel and summation order: results agree to rounding


def _inputs(rng, P, device):
    import torch
    t = lambda a: torch.as_tensor(a.astype(np.float32), device=device)
    x = dict(rgb=t(rng.standard_normal(3 * P)), depth=t(rng.uniform(1, 20, P)), pm=t(rng.standard_normal(3 * P)))
    y = dict(rgb=t(rng.standard_normal(3 * P)), depth=t(rng.uniform(1, 20, P)), pm=t(rng.standard_normal(3 * P)))
    mask = t((rng.uniform(size=P) > 0.25).astype(np.float64))
    return x, y, mask


def test_noalloc_loss_matches_regular_loss_on_two_calls():
    import torch
    from paper_2507_03737_gb300 import binding as B
    from paper_2507_03737_gb300 import scenes
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cams_list = [scenes.camera(61, 23, 50, 50, 30, 11), scenes.camera(40, 70, 60, 60, 20, 35),
                 scenes.camera(17, 9, 20, 20, 8, 4)]
    cams = B.make_cameras(cams_list)
    P = sum(c["width"] * c["height"] for c in cams_list)
    ctx = B.s3gs_create(0)
    rng = np.random.default_rng(1234)
    try:
        for call in range(2):
            x, y, mask = _inputs(rng, P, dev)
            w = (0.98, 0.3 + call, 0.02)
            ref = {k: torch.empty_like(v) for k, v in x.items()}
            got = {k: torch.full_like(v, float("nan")) for k, v in x.items()}
            loss_ref = torch.zeros(1, device=dev)
            loss_got = torch.full((1,), float("nan"), device=dev)
            B.s3gs_mapping_loss(ctx, cams, 3, x["rgb"], x["depth"], x["pm"], y["rgb"], y["depth"], y["pm"], mask,
                                *w, ref["rgb"], ref["depth"], ref["pm"], loss_ref)
            B.s3gs_mapping_loss_noalloc(cams, 3, x["rgb"], x["depth"], x["pm"], y["rgb"], y["depth"], y["pm"], mask,
                                        *w, got["rgb"], got["depth"], got["pm"], loss_got)
            torch.cuda.synchronize()
            lr, lg = float(loss_ref.item()), float(loss_got.item())
            assert np.isfinite(lg) and abs(lg - lr) <= TOL_REL * abs(lr), (call, lr, lg)
            for k in ref:
                a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
                np.testing.assert_allclose(a, b, rtol=TOL_REL, atol=1e-12, err_msg=f"call {call} {k}")
        # sizes beyond the static scratch are rejected with a message
        many = B.make_cameras([cams_list[2]] * 33)
        with pytest.raises(B.S3GSError) as e:
            B.s3gs_mapping_loss_noalloc(many, 33, x["rgb"], None, None, y["rgb"], None, None, None, 1.0, 0.0, 0.0,
                                        None, None, None, loss_got)
        assert e.value.status == B.S3GS_E_INVALID and "static scratch" in str(e.value)
    finally:
        B.s3gs_destroy(ctx)
