"""Pins of the FP64 decode oracle (Sec. III-A, Eq. 1-5) against hand-worked values."""
import json
import math
import os

import numpy as np
import torch

import oracle
from oracle.decode import _bf16_midpoint_distance
from paper_2505_18992_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _val(s):
    return {"ln3": math.log(3.0), "-ln3": -math.log(3.0)}.get(s, None) if isinstance(s, str) and \
        s.endswith("ln3") else float(s)


def _hand_mlp(g):
    k = g["k"]
    mk = {}
    b2s = {"opacity": [_val(x) for x in g["b2_opacity_logits"]],
           "color": [_val(x) for row in g["b2_color_logits"] for x in row],
           "cov": [_val(x) for row in g["b2_cov_logits"] for x in row]}
    for name, dout in (("opacity", k), ("color", 3 * k), ("cov", 7 * k)):
        mk[name] = (np.zeros((32, 36)), np.ones(32), np.zeros((dout, 32)), np.array(b2s[name]))
    return mk


def test_one_anchor_hand_worked():
    with open(os.path.join(GOLDEN, "decode_one_anchor.json")) as fh:
        g = json.load(fh)
    T = np.eye(4)
    T[:3, 3] = -np.array(g["camera_center"])
    out = oracle.decode(np.array([g["anchor"]]), np.zeros((1, 32)), np.array([g["scaling"]]),
                        np.array([g["offsets"]]), _hand_mlp(g), T, 100.0, 100.0, 100.0, 100.0,
                        200, 200)
    e = g["expected"]
    assert out["n"] == e["n_valid"]
    assert out["src_index"].tolist() == e["src_index"]
    assert np.allclose(out["opacities"], e["opacity"], atol=1e-15)
    assert np.allclose(out["colors"], e["color"], atol=1e-15)
    assert np.allclose(out["scales"], e["scale"], atol=1e-15)
    assert np.allclose(out["quats"], e["quat"], atol=1e-15)
    assert np.allclose(out["means"], e["mean"], atol=1e-14)


def test_view_inputs_eq3_reach_the_network():
    # W1 picks the direction and distance inputs (columns 32..35) into hidden units
    # 0..3, W2 copies hidden 0..3 to the cov scale logits of Gaussian 0; with the
    # camera at (1,-1,6) and the anchor at (1,2,10): delta = 5, d = (0, .6, .8)
    k = 1
    W1 = np.zeros((32, 36))
    for i in range(4):
        W1[i, 32 + i] = 1.0
    mlp = {"opacity": (np.zeros((32, 36)), np.ones(32), np.zeros((1, 32)), np.array([1.0])),
           "color": (np.zeros((32, 36)), np.zeros(32), np.zeros((3, 32)), np.zeros(3)),
           "cov": (W1, np.zeros(32), np.zeros((7, 32)), np.array([0, 0, 0, 1.0, 0, 0, 0]))}
    W2 = np.zeros((7, 32))
    W2[0, 1] = 1.0   # -> s_x logit = d_y
    W2[1, 2] = 1.0   # -> s_y logit = d_z
    W2[2, 3] = 0.1   # -> s_z logit = delta / 10
    mlp["cov"] = (W1, np.zeros(32), W2, np.array([0, 0, 0, 1.0, 0, 0, 0]))
    T = np.eye(4)
    T[:3, 3] = -np.array([1.0, -1.0, 6.0])
    out = oracle.decode(np.array([[1.0, 2.0, 10.0]]), np.zeros((1, 32)), np.ones((1, 3)),
                        np.zeros((1, k, 3)), mlp, T, 100.0, 100.0, 100.0, 100.0, 200, 200)
    sig = lambda x: 1 / (1 + math.exp(-x))  # noqa: E731
    assert np.allclose(out["scales"][0], [sig(0.6), sig(0.8), sig(0.5)], atol=1e-15)


def test_frustum_cull_boundaries():
    # camera at the origin looking +z, 100x100, f = 100, centre (50,50): the kept
    # band is u in [-15, 115]  <=>  x/z in [-0.65, 0.65]
    z = 4.0
    xs = np.array([0.0, 0.64, 0.66, -0.64, -0.66]) * z
    anchors = np.stack([xs, np.zeros(5), np.full(5, z)], 1)
    anchors = np.concatenate([anchors, [[0, 0, 0.19], [0, 0, 0.21]]])
    mlp = {"opacity": (np.zeros((32, 36)), np.ones(32), np.zeros((1, 32)), np.array([1.0])),
           "color": (np.zeros((32, 36)), np.zeros(32), np.zeros((3, 32)), np.zeros(3)),
           "cov": (np.zeros((32, 36)), np.zeros(32), np.zeros((7, 32)), np.array([0, 0, 0, 1.0, 0, 0, 0]))}
    out = oracle.decode(anchors, np.zeros((7, 32)), np.ones((7, 3)), np.zeros((7, 1, 3)), mlp,
                        np.eye(4), 100.0, 100.0, 50.0, 50.0, 100, 100)
    assert out["keep"].tolist() == [True, True, False, True, False, False, True]
    assert out["src_index"].tolist() == [0, 1, 3, 6]


def test_bf16_rounding_hand_values():
    vals = torch.tensor([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -3.0 - 2 ** -7, 1e-3],
                        dtype=torch.float64)
    r = oracle.bf16_round(vals).detach().numpy()
    # ties go to even: 1+2^-8 -> 1; 1+3*2^-8 -> 1+2^-6; 1+2^-7 exact; -3-2^-7 is a tie -> -3
    assert r[0] == 1.0 and r[1] == 1.0 + 2 ** -6 and r[2] == 1.0 + 2 ** -7 and r[3] == -3.0
    # 1e-3 = 0x3A83126F in fp32 -> bf16 0x3A83 = 0.00099945068359375
    assert r[4] == 0.00099945068359375
    d = _bf16_midpoint_distance(np.array([1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.0 + 2 ** -8]))
    assert d[0] == 0.0 and d[1] == 2 ** -8 and d[2] == 2 ** -8  # midpoints of [3, 3+2^-6] at 3+2^-7


def test_bf16_decode_is_exact_on_bf16_representable_networks():
    # every weight, input and hidden value is a small dyadic number, so BF16
    # rounding is the identity and the BF16 decode must equal the FP64 one
    rng = np.random.default_rng(5)
    A, k = 7, 3
    feats = rng.integers(-4, 5, size=(A, 32)) / 4.0
    mlp = {}
    for name, dout in (("opacity", k), ("color", 3 * k), ("cov", 7 * k)):
        W1 = rng.integers(-2, 3, size=(32, 36)) / 8.0
        W1[:, 32:] = 0.0
        mlp[name] = (W1, rng.integers(-4, 5, size=32) / 8.0,
                     rng.integers(-2, 3, size=(dout, 32)) / 64.0, rng.integers(-4, 5, size=dout) / 8.0)
    anchors = np.stack([rng.uniform(-1, 1, A), rng.uniform(-1, 1, A), rng.uniform(3, 5, A)], 1)
    args = (anchors, feats, np.full((A, 3), 0.25), rng.uniform(-1, 1, (A, k, 3)), mlp, np.eye(4),
            100.0, 100.0, 50.0, 50.0, 100, 100)
    a = oracle.decode(*args)
    b = oracle.decode(*args, bf16=True)
    assert a["n"] == b["n"] and a["n"] > 0
    for key in ("means", "scales", "quats", "opacities", "colors"):
        assert np.array_equal(a[key], b[key]), key


def test_parameter_count_of_the_stated_architecture():
    # three 36->32->{k,3k,7k} MLPs at k = 10: 7,182 parameters (the paper's table
    # prints 0.003M, which this architecture cannot give)
    assert oracle.n_mlp_params(10) == 7182


def test_decode_gradients_central_differences():
    sc = scenes.street_anchors(n_anchors=4, length=2.0, width=200, height=100, f=100.0, k=2,
                               cam_x=-3.0)
    sc.offsets = sc.offsets.astype(np.float64)
    rng = np.random.default_rng(9)
    base = oracle.decode_scene(sc)
    assert base["n"] >= 2
    g = {"means": rng.normal(size=(base["n"], 3)), "scales": rng.normal(size=(base["n"], 3)),
         "quats": rng.normal(size=(base["n"], 4)), "opacities": rng.normal(size=base["n"]),
         "colors": rng.normal(size=(base["n"], 3))}
    out = oracle.decode_scene(sc, grads=g)

    def loss(feat=None, off=None, scal=None, mlp=None):
        cam = sc.camera
        r = oracle.decode(sc.anchors, sc.features if feat is None else feat,
                          sc.scaling if scal is None else scal, sc.offsets if off is None else off,
                          sc.mlp if mlp is None else mlp, cam.T_cw[0], cam.fx, cam.fy, cam.cx,
                          cam.cy, cam.width, cam.height)
        assert np.array_equal(r["src_index"], base["src_index"])
        return sum((r[key] * g[key]).sum() for key in g)

    h = 1e-6

    def check(arr, grad, make):
        arr = np.asarray(arr, np.float64)
        for idx in np.ndindex(arr.shape):
            p, m = arr.copy(), arr.copy()
            p[idx] += h
            m[idx] -= h
            fd = (make(p) - make(m)) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, grad[idx])

    check(sc.features, out["d_features"], lambda a: loss(feat=a))
    check(sc.offsets, out["d_offsets"], lambda a: loss(off=a))
    check(sc.scaling, out["d_scaling"], lambda a: loss(scal=a))
    flat = oracle.flatten_mlp(sc.mlp)
    pick = np.random.default_rng(1).choice(flat.size, 400, replace=False)

    def unflat(vec):
        mk, pos = {}, 0
        for name in oracle.MLP_ORDER:
            parts = []
            for prm in sc.mlp[name]:
                parts.append(vec[pos:pos + prm.size].reshape(prm.shape))
                pos += prm.size
            mk[name] = tuple(parts)
        return mk

    for i in pick:
        p, m = flat.copy(), flat.copy()
        p[i] += h
        m[i] -= h
        fd = (loss(mlp=unflat(p)) - loss(mlp=unflat(m))) / (2 * h)
        assert abs(fd - out["d_w"][i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, out["d_w"][i])
