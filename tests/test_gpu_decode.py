"""GPU anchor decoder (FP32 and BF16 tensor-core forms) against the FP64 oracle."""
import copy
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2505_18992_gb300 import scenes
from paper_2505_18992_gb300 import vpgs as C
from paper_2505_18992_gb300.decode import Decoder
from tests.helpers import assert_grad_close, dev

pytestmark = pytest.mark.gpu

OUT_KEYS = ("means", "scales", "quats", "opacities", "colors")


def _street(n=3000, seed=2, length=30.0):
    return scenes.street_anchors(n_anchors=n, length=length, seed=seed)


def _oracle(sc, bf16, grads=None):
    cam = sc.camera
    return oracle.decode(sc.anchors, sc.features, sc.scaling, sc.offsets, sc.mlp, cam.T_cw[0], cam.fx,
                         cam.fy, cam.cx, cam.cy, cam.width, cam.height, bf16=bf16, grads=grads)


def _gpu(sc, bf16, features_bf16=False):
    d = Decoder(sc.k, bf16=bf16)
    feats = dev(sc.features)
    if features_bf16:
        feats = feats.to(torch.bfloat16).contiguous()
    T = dev(sc.camera.T_cw[0], torch.float64)
    out = d.forward(dev(sc.anchors), feats, dev(sc.scaling), dev(sc.offsets), dev(oracle.flatten_mlp(sc.mlp)),
                    sc.camera, T)
    torch.cuda.synchronize()
    return d, feats, T, out


def _compare_outputs(out, ref, flags, k, atol):
    n = int(out["n"])
    src = out["src_index"][:n].cpu().numpy()
    flagged_anchor = flags[src // k]
    ref_src = ref["src_index"]
    # the valid set and its order agree away from flagged anchors
    keep_gpu = src[~flagged_anchor]
    keep_ref = ref_src[~flags[ref_src // k]]
    assert np.array_equal(keep_gpu, keep_ref)
    pos_ref = {int(s): i for i, s in enumerate(ref_src)}
    gi = np.nonzero(~flagged_anchor)[0]
    ri = np.array([pos_ref[int(s)] for s in src[gi]])
    for key in OUT_KEYS:
        g = out[key][:n].cpu().numpy()[gi]
        r = ref[key][ri]
        assert np.abs(g - r).max() <= atol, (key, float(np.abs(g - r).max()))
    return gi, ri


@pytest.mark.parametrize("bf16", [False, True])
def test_decode_forward_parity(bf16):
    sc = _street()
    ref = _oracle(sc, bf16)
    _, _, _, out = _gpu(sc, bf16)
    assert ref["n"] > 1000
    assert ref["flags"].mean() < (0.15 if bf16 else 0.02)
    _compare_outputs(out, ref, ref["flags"], sc.k, 1e-5)


def test_decode_bf16_features_input():
    sc = _street(n=1500, seed=4)
    sc.features = torch.tensor(sc.features).to(torch.bfloat16).to(torch.float32).numpy()
    ref = _oracle(sc, True)
    _, _, _, out = _gpu(sc, True, features_bf16=True)
    _compare_outputs(out, ref, ref["flags"], sc.k, 1e-5)


@pytest.mark.parametrize("bf16", [False, True])
def test_decode_backward_parity(bf16):
    _backward_parity(_street(n=2000, seed=6), bf16)


@pytest.mark.parametrize("k", [1, 4, 7])
@pytest.mark.parametrize("bf16", [False, True])
def test_decode_other_gaussians_per_anchor(bf16, k):
    """k below 10: the heads' outputs (k, 3k, 7k) pad to the tensor-core tiles
    differently; forward and backward still match the oracle."""
    sc = scenes.street_anchors(n_anchors=1500, length=20.0, seed=9, k=k)
    ref = _oracle(sc, bf16)
    _, _, _, out = _gpu(sc, bf16)
    assert ref["n"] > (20 if k == 1 else 1000)  # one Gaussian an anchor: few survive
    assert ref["flags"].mean() < (0.15 if bf16 else 0.02)
    _compare_outputs(out, ref, ref["flags"], sc.k, 1e-5)
    _backward_parity(sc, bf16)


def _in_view_subset(n):
    """The first n anchors of a street scene that decode to at least one
    Gaussian (so that few-anchor cases still have outputs to compare)."""
    sc0 = _street(n=2000, seed=2)
    ref0 = _oracle(sc0, True)
    sel = np.unique(ref0["src_index"] // sc0.k)[:n]
    sc = copy.copy(sc0)
    sc.anchors, sc.features = sc0.anchors[sel].copy(), sc0.features[sel].copy()
    sc.scaling, sc.offsets = sc0.scaling[sel].copy(), sc0.offsets[sel].copy()
    return sc


@pytest.mark.parametrize("n", [1, 63, 64, 65, 130])
@pytest.mark.parametrize("bf16", [False, True])
def test_decode_few_anchors(bf16, n):
    """Fewer 64-anchor chunks than resident forward blocks (most blocks find no
    chunk and leave) and a ragged last chunk; a second call on the same decoder
    starts its chunk tickets from zero again and gives the same outputs."""
    sc = _in_view_subset(n)
    ref = _oracle(sc, bf16)
    assert ref["n"] >= 1
    d, feats, T, out = _gpu(sc, bf16)
    _compare_outputs(out, ref, ref["flags"], sc.k, 1e-5)
    first = {k: out[k][: int(out["n"])].clone() for k in OUT_KEYS}
    out2 = d.forward(dev(sc.anchors), feats, dev(sc.scaling), dev(sc.offsets), dev(oracle.flatten_mlp(sc.mlp)),
                     sc.camera, T)
    torch.cuda.synchronize()
    assert int(out2["n"]) == int(out["n"])
    for k in OUT_KEYS:
        assert torch.equal(out2[k][: int(out2["n"])], first[k]), k


def _backward_parity(sc, bf16):
    ref0 = _oracle(sc, bf16)
    rng = np.random.default_rng(3)
    n = ref0["n"]
    # upstream gradients; zero them on Gaussians of flagged anchors so that both
    # sides ignore decisions taken at a margin
    keep = ~ref0["flags"][ref0["src_index"] // sc.k]
    g = {"means": rng.normal(size=(n, 3)), "scales": rng.normal(size=(n, 3)),
         "quats": rng.normal(size=(n, 4)), "opacities": rng.normal(size=n), "colors": rng.normal(size=(n, 3))}
    for key in g:
        g[key][~keep] = 0.0
    ref = _oracle(sc, bf16, grads=g)
    d, feats, T, out = _gpu(sc, bf16)
    m = int(out["n"])
    src = out["src_index"][:m].cpu().numpy()
    pos_ref = {int(s): i for i, s in enumerate(ref["src_index"])}
    idx = np.array([pos_ref.get(int(s), -1) for s in src])
    gg = {}
    for key in OUT_KEYS:
        arr = np.zeros((out[key].shape[0],) + g[key].shape[1:], np.float32)
        ok = idx >= 0
        arr[:m][ok] = g[key][idx[ok]]
        gg[key] = dev(arr)
    res = d.backward(dev(sc.anchors), feats, dev(sc.scaling), dev(sc.offsets),
                     dev(oracle.flatten_mlp(sc.mlp)), sc.camera, T, out, gg)
    torch.cuda.synchronize()
    assert_grad_close(res["features"].cpu().numpy(), ref["d_features"], "features")
    assert_grad_close(res["offsets"].cpu().numpy(), ref["d_offsets"], "offsets")
    assert_grad_close(res["scaling"].cpu().numpy(), ref["d_scaling"], "scaling")
    assert_grad_close(res["params"].cpu().numpy(), ref["d_w"], "mlp params")


def test_decode_then_render_uses_the_device_count():
    from paper_2505_18992_gb300.render import Intrinsics, Renderer
    sc = _street(n=2000, seed=8)
    _, _, T, out = _gpu(sc, False)
    cam = sc.camera
    r = Renderer(Intrinsics(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy))
    img = r.forward(out["means"], out["scales"], out["quats"], out["opacities"], out["colors"],
                    T[None].contiguous(), n_dev=out["n_dev"])
    n = int(out["n"])
    img2 = r.forward(out["means"][:n].contiguous(), out["scales"][:n].contiguous(),
                     out["quats"][:n].contiguous(), out["opacities"][:n].contiguous(),
                     out["colors"][:n].contiguous(), T[None].contiguous())
    for k in ("rgb", "depth", "alpha", "n_contrib"):
        assert torch.equal(img[k], img2[k]), k


def test_decode_rejects_bad_arguments():
    a = C.vpgs_anchors(None, None, None, None, 10, 11, 0)  # k > 10
    mlp = C.vpgs_mlp(None, 0)
    cam = C.vpgs_camera(100, 100, 100.0, 100.0, 50.0, 50.0)
    opts = C.vpgs_decode_opts(0.2, 0.15)
    out = C.vpgs_gaussian_buffers()
    code = C.vpgs_decode_anchors(None, 0, ctypes.byref(a), ctypes.byref(mlp), ctypes.byref(cam), None,
                                 ctypes.byref(opts), ctypes.byref(out), None, None, None)
    assert code == 1


@pytest.mark.parametrize("bf16", [False, True])
def test_full_size_street_decode(bf16):
    # 100,000 anchors, 1241x376 camera: the decode the benchmark times
    sc = scenes.street_anchors()
    ref = _oracle(sc, bf16)
    _, _, _, out = _gpu(sc, bf16)
    assert int(out["n"]) > 400_000
    assert ref["flags"].mean() < (0.15 if bf16 else 0.02)
    _compare_outputs(out, ref, ref["flags"], sc.k, 1e-5)
