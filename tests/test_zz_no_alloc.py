"""The allocation-free scoring entry point against the regular one.

voldor_score_records_noalloc serves callers that cannot allocate device
memory (inside a graph capture, under a fixed memory budget, or with their own
allocator). It must give the same dense scores as voldor_score_hypotheses,
call after call, although all its calls share one scratch array.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from tests.helpers import f32_hypotheses, f32_state, small_window

pytestmark = pytest.mark.gpu


def _records(w, depth, rig, poses, t, p):
    """Pixel records of frame t in the layout the header documents (FP64
    geometry, FP32 storage); pixels whose pi_{t-1} leaves the image or lies
    behind camera t-1 are left out."""
    fx, fy, cx, cy = w.K
    H, W = depth.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    th = depth.astype(np.float64)
    P0 = np.stack([th * (xs - cx) / fx, th * (ys - cy) / fy, th], -1).reshape(-1, 3)
    C = np.eye(4)
    for i in range(t - 1):
        C = poses[i] @ C
    P = P0 @ C[:3, :3].T + C[:3, 3]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * P[:, 0] / P[:, 2] + cx
        v = fy * P[:, 1] / P[:, 2] + cy
    if t == 1:
        u, v = xs.ravel(), ys.ravel()
    ok = (P[:, 2] > 0) & (u >= 0) & (u <= W - 1) & (v >= 0) & (v <= H - 1)
    P, u, v = P[ok], u[ok], v[ok]
    x0 = np.minimum(np.floor(u).astype(int), W - 2)
    y0 = np.minimum(np.floor(v).astype(int), H - 2)
    ax, ay = u - x0, v - y0
    F = w.flows[t - 1].astype(np.float32).astype(np.float64)
    fl = ((1 - ax) * (1 - ay))[:, None] * F[y0, x0] + (ax * (1 - ay))[:, None] * F[y0, x0 + 1] \
        + ((1 - ax) * ay)[:, None] * F[y0 + 1, x0] + (ax * ay)[:, None] * F[y0 + 1, x0 + 1]
    n = np.linalg.norm(fl, axis=1)
    log2_alpha = np.log2(p.a1) + p.a2 * n / np.log(2.0)
    beta = np.maximum(p.b1 * n + p.b2, p.beta_min)
    xmu = np.clip(p.lambda_ ** 2 * n * n, p.x_min, p.x_max)
    ysm = 2.0 ** -np.abs(beta * (np.log2(xmu) - log2_alpha))
    mu_over_beta = ysm / (xmu * (1 + ysm) ** 2)
    rec = np.zeros((len(P), 12))
    rec[:, 0] = P[:, 0] / P[:, 2]
    rec[:, 1] = fy / fx * P[:, 1] / P[:, 2]
    rec[:, 2] = 1.0 / P[:, 2]
    rec[:, 3] = fl[:, 0] / fx
    rec[:, 4] = fl[:, 1] / fx
    rec[:, 5] = beta
    rec[:, 6] = beta * (np.log2(fx * fx) - log2_alpha)
    rec[:, 7] = fx * fx * mu_over_beta
    rec[:, 8] = rig[t - 1].ravel()[ok]
    return rec.astype(np.float32)


def test_noalloc_scores_match_the_context_entry_point():
    torch = pytest.importorskip("torch")
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    w = small_window(seed=1000)
    rng = np.random.default_rng(77)
    depth, rig = f32_state(rng, w)
    p = voldor.default_params(hyps_per_frame=256, inv_depth_min=w.inv_depth_range[0],
                              inv_depth_max=w.inv_depth_range[1])
    g = voldor.Window(w.flows.astype(np.float32), w.K, p)
    g.set_state(poses=w.poses, depth=depth, rigidness=rig, iteration=0)
    fx = w.K[0]
    for t in (1, 3):
        R, tv = f32_hypotheses(rng, w.poses[t - 1][:3, :3], w.poses[t - 1][:3, 3], 200)
        L_ref = g.score_hypotheses(t, R, tv)
        rec = torch.from_numpy(_records(w, depth, rig, w.poses, t, p)).cuda()
        hyp = np.concatenate([(R - np.eye(3)).reshape(-1, 9), tv], 1).astype(np.float32)   # fx == fy
        hyp = torch.from_numpy(hyp).cuda()
        for _ in range(2):                       # two calls in a row share the scratch array
            L = torch.full((len(R),), float("nan"), dtype=torch.float64, device="cuda")
            voldor.score_records_noalloc(rec, hyp, L, p.x_min / fx ** 2, p.x_max / fx ** 2)
            torch.cuda.synchronize()
            got = L.cpu().numpy()
            rel = np.abs(got - L_ref) / np.abs(L_ref)
            assert rel.max() < 1e-5, rel.max()
    g.destroy()


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    rec = torch.zeros((4, 12), dtype=torch.float32, device="cuda")
    hyp = torch.zeros((8193, 12), dtype=torch.float32, device="cuda")
    L = torch.zeros(8193, dtype=torch.float64, device="cuda")
    with pytest.raises(voldor.VoldorError) as e:
        voldor.score_records_noalloc(rec, hyp, L, 1e-12, 1.0)
    assert e.value.status == voldor.ERR_INVALID_ARG


def test_noalloc_rejects_misaligned_pointers_and_bad_tensors():
    """A records pointer off the 16-byte boundary (a tensor sliced by one
    float) is refused on the host before any device work; the Python wrapper
    refuses a wrong dtype, width or a short L."""
    import ctypes
    torch = pytest.importorskip("torch")
    from paper_2104_06789_gb300 import build, voldor
    build.build()
    flat = torch.zeros(13 * 4, dtype=torch.float32, device="cuda")
    hyp = torch.zeros((2, 12), dtype=torch.float32, device="cuda")
    L = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = voldor.lib().voldor_score_records_noalloc(ctypes.c_void_p(flat.data_ptr() + 4), 4,
                                                  ctypes.c_void_p(hyp.data_ptr()), 2, ctypes.c_double(1e-12),
                                                  ctypes.c_double(1.0), ctypes.c_void_p(L.data_ptr()),
                                                  ctypes.c_void_p(0))
    assert st == voldor.ERR_INVALID_ARG
    rec = torch.zeros((4, 12), dtype=torch.float32, device="cuda")
    for bad in (dict(records=rec.double()), dict(records=rec[:, :9].contiguous()), dict(L=L[:1])):
        args = dict(records=rec, hyps=hyp, L=L)
        args.update(bad)
        with pytest.raises(ValueError):
            voldor.score_records_noalloc(args["records"], args["hyps"], args["L"], 1e-12, 1.0)
    torch.cuda.synchronize()
