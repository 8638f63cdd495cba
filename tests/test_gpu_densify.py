"""Densification and pruning on the GPU against the FP64 oracle: the same
decisions (bit-exact output order and source of every output), copies
bit-exact, split children's means within FP32 rounding of the oracle's FP64
value and their log-scales exact, moments carried or zeroed as specified,
padding zero, overflow reported; and the chain rule's densification
statistic equal to |dL/d(u, v)| in NDC from the oracle's gradient."""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic as S
from parity_helpers import MARGIN_FLAG, gpu_view, oracle_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_16728_b300 as gsr  # noqa: E402
from paper_2311_16728_b300 import _lib as L  # noqa: E402

THR = np.float32(2e-4)
LOGIT_MIN = np.float32(np.log(0.005 / 0.995))
SPLIT = np.float32(np.log(0.03))
SHRINK = np.float32(np.log(1.6))


def _flat(G, n):
    return np.concatenate([G.mean_op.cpu().numpy()[:n], G.quat.cpu().numpy()[:n], G.logscale.cpu().numpy()[:n],
                           G.sh.cpu().numpy()[:, :n].transpose(1, 0, 2).reshape(n, 48)], 1)


def _run(p, stat, count, eps, cap, m=None, v=None):
    n = p.n
    g = gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh)
    m = m if m is not None else g.zeros_like()
    v = v if v is not None else g.zeros_like()
    out, om, ov = gsr.Gaussians.zeros(cap), gsr.Gaussians.zeros(cap), gsr.Gaussians.zeros(cap)
    for t in out.tensors() + om.tensors() + ov.tensors():
        t.fill_(7.0)  # the padding must overwrite this
    cfg = L.gsr_densify_config(float(THR), float(LOGIT_MIN), float(SPLIT), float(SHRINK))
    sz = ctypes.c_size_t()
    L.gsr_densify_workspace_size(n, ctypes.byref(sz))
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    ts, tc, te = dev(stat), dev(count), dev(eps)
    pb = [x.buffers_struct() for x in (g, m, v, out, om, ov)]
    L.gsr_densify(ctypes.byref(pb[0]), ctypes.byref(pb[1]), ctypes.byref(pb[2]), n, ts.data_ptr(), tc.data_ptr(),
                  te.data_ptr(), ctypes.byref(cfg), ctypes.byref(pb[3]), ctypes.byref(pb[4]), ctypes.byref(pb[5]),
                  cap, d_n.data_ptr(), ws.data_ptr(), ws.numel(), st.data_ptr(), None)
    torch.cuda.synchronize()
    return g, m, v, out, om, ov, int(d_n.item()), int(st.item())


def _case(n=6000, seed=0):
    rng = np.random.default_rng(seed)
    p = S.room_scene(n, seed=seed)
    p.mean_op[:, 3] = rng.normal(-2.0, 2.5, n).astype(np.float32)  # many below the prune bound
    p.logscale[:, :3] = rng.normal(-3.8, 0.5, (n, 3)).astype(np.float32)
    p.quat[rng.random(n) < 0.05] = 0.0  # some empty slots
    count = rng.integers(0, 6, n).astype(np.float32)
    stat = (count * rng.lognormal(np.log(2e-4), 1.0, n)).astype(np.float32)
    eps = rng.standard_normal((n, 6)).astype(np.float32)
    return p, stat, count, eps


def test_densify_matches_oracle():
    p, stat, count, eps = _case()
    n = p.n
    rng = np.random.default_rng(9)
    g0 = gsr.Gaussians.from_arrays(p.mean_op, p.quat, p.logscale, p.sh)
    m = gsr.Gaussians.from_arrays(*(rng.standard_normal(t.shape).astype(np.float32) for t in
                                    (p.mean_op, p.quat, p.logscale, p.sh)))
    v = gsr.Gaussians.from_arrays(*(rng.random(t.shape).astype(np.float32) for t in
                                    (p.mean_op, p.quat, p.logscale, p.sh)))
    g, m, v, out, om, ov, n_out, st = _run(p, stat, count, eps, 2 * n, m, v)
    ref = oracle.densify(p.mean_op, p.quat, p.logscale, stat, count, eps, THR, LOGIT_MIN, SPLIT, SHRINK)
    kinds = np.bincount(ref["kind"], minlength=4)
    print(f"n {n} -> {n_out}: kept/clone originals {kinds[0]}, clone copies {kinds[1]}, split children "
          f"{kinds[2] + kinds[3]}, pruned or empty {n - kinds[0] - kinds[2]}")
    assert st == 0 and n_out == len(ref["src"])
    assert min(kinds[1], kinds[2]) > 50 and n - kinds[0] - kinds[2] > 50  # every branch exercised
    src, kind = ref["src"], ref["kind"]
    P_in, P_out = _flat(g, n), _flat(out, n_out)
    M_in, M_out, V_in, V_out = _flat(m, n), _flat(om, n_out), _flat(v, n), _flat(ov, n_out)
    split = kind >= 2
    # copies and carried fields bit-exact
    assert np.array_equal(P_out[~split], P_in[src[~split]])
    assert np.array_equal(P_out[split][:, 3:8], P_in[src[split]][:, 3:8])    # opacity, rotation
    assert np.array_equal(P_out[split][:, 12:], P_in[src[split]][:, 12:])    # SH
    assert np.array_equal(P_out[split][:, 8:11].astype(np.float64), ref["logscale"][split])
    # split means within FP32 rounding of the FP64 oracle
    scale = np.abs(P_in[src[split]][:, 0:3]).max(1, keepdims=True) + np.exp(P_in[src[split]][:, 8:11]).max(1, keepdims=True) * 4
    err = np.abs(P_out[split][:, 0:3] - ref["mean"][split])
    assert (err <= 4e-7 * scale).all(), (err / scale).max()
    # moments: survivors keep theirs, new Gaussians start at zero
    keep = kind == 0
    assert np.array_equal(M_out[keep], M_in[src[keep]]) and np.array_equal(V_out[keep], V_in[src[keep]])
    assert (M_out[~keep] == 0).all() and (V_out[~keep] == 0).all()
    # padding
    for t in out.tensors() + om.tensors() + ov.tensors():
        tail = t[n_out:] if t.dim() == 2 else t[:, n_out:]
        assert (tail == 0).all()


def test_densify_overflow_is_reported():
    p, stat, count, eps = _case(2000, seed=3)
    ref = oracle.densify(p.mean_op, p.quat, p.logscale, stat, count, eps, THR, LOGIT_MIN, SPLIT, SHRINK)
    cap = len(ref["src"]) - 10
    *_, n_out, st = _run(p, stat, count, eps, cap)
    assert st & (1 << L.GSR_ERR_CAPACITY) and n_out == len(ref["src"])


def test_densify_statistic_is_the_ndc_gradient_norm():
    p, cam = S.perturb(S.tiny_scene()), S.tiny_camera()
    vb, g = gpu_view(p, cam)
    ca = cam.as_array()
    dec = oracle.decide(p.mean_op, p.quat, p.logscale, ca, cam.width, cam.height)
    sc = oracle_scene(p)
    img, T, nc, mg = oracle.render(sc, ca, cam.width, cam.height, dec)
    dimg = S.random_grad_image(3, cam.height, cam.width, seed=4)
    dimg[:, mg < MARGIN_FLAG] = 0.0
    _, g2ref = oracle.render_bwd(sc, ca, cam.width, cam.height, dec, dimg.astype(np.float64))
    stat = torch.zeros(p.n, device="cuda")
    count = torch.zeros(p.n, device="cuda")
    grads = g.zeros_like()
    vb.render_bwd(g, grads, dimg=torch.tensor(dimg, device="cuda"), densify_stat=stat, densify_count=count)
    torch.cuda.synchronize()
    ref = np.hypot(g2ref[:, 0] * cam.width / 2, g2ref[:, 1] * cam.height / 2)
    vis = dec.visible > 0
    assert np.array_equal(count.cpu().numpy(), vis.astype(np.float32))
    got = stat.cpu().numpy()
    assert np.allclose(got[vis], ref[vis], rtol=1e-3, atol=1e-6 * ref.max())
    assert (got[~vis] == 0).all()
