"""GPU parity of the space-variant extension (Section 4: each pixel averages
over its own box or hat) against the FP64 oracle, element by element, within
0.05 gray levels; ragged sizes, every table size (r_max up to 4, 8, 16 for the
box, 4 and 8 for the hat), the degenerate radius 0, clamped radii, u8 input,
and a full-size image on sampled pixels."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 0.05


@pytest.fixture(scope="module")
def bf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_4204_gb300 import build
    build.build()
    import paper_1105_4204_gb300 as pkg
    return pkg


def _sv(bf, img, rad, plan, r_max, spatial="box"):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    rt = torch.from_numpy(np.ascontiguousarray(rad, dtype=np.int32)).cuda()
    out = bf.forward_space_variant(plan, t, rt, r_max=r_max, spatial=spatial)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("H,W", [(1, 1), (1, 17), (5, 3), (37, 53), (70, 131), (97, 64)])
@pytest.mark.parametrize("r_max", [0, 3, 8, 13, 16])
def test_random_radius_maps(bf, oracle, H, W, r_max):
    img = synth.rectangles(H, W, n_rect=5, noise=10.0, seed=H * 100 + W)
    rad = synth.radius_map(H, W, r_max, seed=r_max, smooth=False)
    plan = bf.Plan(3.0, 25.0, kind="box")
    out = _sv(bf, img, rad, plan, r_max)
    ref = oracle.bf_brute_sv(img, rad, sigma_r=25.0, r_max=r_max, N=plan.N)
    err = np.abs(out - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("sigma_r,N", [(10.0, 264), (20.0, 66), (60.0, 8), (200.0, 1)])
def test_degrees(bf, oracle, sigma_r, N):
    img = synth.smooth_field(75, 88, noise=5.0, seed=int(sigma_r))
    rad = synth.radius_map(75, 88, 8, seed=3)
    plan = bf.Plan(2.0, sigma_r, kind="gauss")
    assert plan.N == N
    out = _sv(bf, img, rad, plan, 8)
    ref = oracle.bf_brute_sv(img, rad, sigma_r=sigma_r, r_max=8, N=N)
    assert np.abs(out - ref).max() <= TOL


def test_radius_zero_returns_the_image(bf):
    img = synth.rectangles(40, 70, noise=10.0, seed=2)
    out = _sv(bf, img, np.zeros(img.shape, np.int32), bf.Plan(3.0, 30.0), 0)
    np.testing.assert_allclose(out, img, rtol=0, atol=1e-4)


def test_constant_radius_is_the_one_box_filter(bf, oracle):
    img = synth.smooth_field(66, 99, noise=5.0, seed=4)
    plan = bf.Plan(3.0, 20.0, kind="box")
    for r0 in (1, 5, 16):
        out = _sv(bf, img, np.full(img.shape, r0, np.int32), plan, 16)
        w1 = oracle.spatial_w1("box", 1.0, radius=r0, passes=1)
        ref = oracle.bf_brute(img, sigma_r=20.0, w1=w1, N=plan.N)
        assert np.abs(out - ref).max() <= TOL


def test_radii_are_clamped_and_u8_matches_f32(bf):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(61, 77)).astype(np.uint8)
    rad = synth.radius_map(61, 77, 6, seed=8, smooth=False)
    plan = bf.Plan(2.0, 30.0)
    a = _sv(bf, img, rad, plan, 6)
    np.testing.assert_array_equal(a, _sv(bf, img.astype(np.float32), rad, plan, 6))
    wild = rad.copy()
    wild[::3] += 40
    wild[1::3] -= 40
    np.testing.assert_array_equal(_sv(bf, img, wild, plan, 6),
                                  _sv(bf, img, np.clip(wild, 0, 6), plan, 6))
    # the same filter with a larger table: the halo, the tile and the
    # fixed-point steps change, so the results agree to rounding
    assert np.abs(a - _sv(bf, img, rad, plan, 16)).max() <= 1e-3


def test_full_size_sampled_and_deterministic(bf, oracle):
    # 2048 x 2048 smooth field, smooth radius map in [0, 8], sigma_r = 20 (N = 66)
    H = W = 2048
    img = synth.smooth_field(H, W, noise=5.0, seed=0)
    rad = synth.radius_map(H, W, 8, seed=1)
    plan = bf.Plan(2.0, 20.0, kind="box")
    out = _sv(bf, img, rad, plan, 8)
    again = _sv(bf, img, rad, plan, 8)
    np.testing.assert_array_equal(out, again)
    idx = synth.sample_indices(H, W, 2048, seed=5)
    ref = oracle.bf_brute_sv_at(img, rad, idx, 8, sigma_r=20.0, N=plan.N)
    err = np.abs(out.ravel()[idx] - ref).max()
    print("space-variant 2048^2 max abs err %.3e over %d px" % (err, len(idx)))
    assert err <= TOL


@pytest.mark.parametrize("coefs", [
    np.array([1.0] + [2.0 * (1.0 - n / 7.0) for n in range(1, 7)]) / 7.0,  # Fejer, N = 6
    np.array([1.0, 0.8, 0.5, 0.3, 0.1]),
])
def test_general_cosine_kernel(bf, oracle, coefs):
    # Section 2.2's general kernel through the space-variant path
    import math
    gamma = math.pi / 510
    img = synth.rectangles(58, 91, n_rect=6, noise=10.0, seed=13)
    rad = synth.radius_map(58, 91, 12, seed=14, smooth=False)
    plan = bf.Plan.cosine(2.0, gamma, coefs, kind="box")
    out = _sv(bf, img, rad, plan, 12)
    ref = oracle.bf_brute_sv_cos(img, rad, gamma, coefs, r_max=12)
    assert np.abs(out - ref).max() <= TOL


# ------------------------------------------------------------------ the hat

@pytest.mark.parametrize("H,W", [(1, 1), (1, 17), (5, 3), (37, 53), (70, 131), (97, 64)])
@pytest.mark.parametrize("r_max", [0, 3, 6, 8])
def test_hat_random_radius_maps(bf, oracle, H, W, r_max):
    img = synth.rectangles(H, W, n_rect=5, noise=10.0, seed=H * 100 + W + 1)
    rad = synth.radius_map(H, W, r_max, seed=r_max + 20, smooth=False)
    plan = bf.Plan(3.0, 25.0, kind="box")
    out = _sv(bf, img, rad, plan, r_max, spatial="hat")
    ref = oracle.bf_brute_sv(img, rad, sigma_r=25.0, r_max=r_max, N=plan.N, spatial="hat")
    err = np.abs(out - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("sigma_r,N", [(10.0, 264), (60.0, 8)])
def test_hat_degrees_and_constant_radius(bf, oracle, sigma_r, N):
    img = synth.smooth_field(75, 88, noise=5.0, seed=int(sigma_r) + 3)
    plan = bf.Plan(2.0, sigma_r, kind="gauss")
    assert plan.N == N
    rad = synth.radius_map(75, 88, 8, seed=5)
    out = _sv(bf, img, rad, plan, 8, spatial="hat")
    ref = oracle.bf_brute_sv(img, rad, sigma_r=sigma_r, r_max=8, N=N, spatial="hat")
    assert np.abs(out - ref).max() <= TOL
    # a constant half-width is the plain filter with separable triangle taps
    for r0 in (1, 8):
        k = np.arange(-r0, r0 + 1)
        w1 = (r0 + 1 - np.abs(k)) / float((r0 + 1) ** 2)
        out = _sv(bf, img, np.full(img.shape, r0, np.int32), plan, 8, spatial="hat")
        ref = oracle.bf_brute(img, sigma_r=sigma_r, w1=w1, N=N)
        assert np.abs(out - ref).max() <= TOL


def test_hat_radius_zero_u8_and_clamping(bf):
    img = synth.rectangles(40, 70, noise=10.0, seed=3)
    plan = bf.Plan(3.0, 30.0)
    out = _sv(bf, img, np.zeros(img.shape, np.int32), plan, 0, spatial="hat")
    np.testing.assert_allclose(out, img, rtol=0, atol=1e-4)
    rng = np.random.default_rng(9)
    u8 = rng.integers(0, 256, size=(61, 77)).astype(np.uint8)
    rad = synth.radius_map(61, 77, 6, seed=10, smooth=False)
    a = _sv(bf, u8, rad, plan, 6, spatial="hat")
    np.testing.assert_array_equal(a, _sv(bf, u8.astype(np.float32), rad, plan, 6, spatial="hat"))
    wild = rad.copy()
    wild[::2] += 30
    np.testing.assert_array_equal(_sv(bf, u8, wild, plan, 6, spatial="hat"),
                                  _sv(bf, u8, np.clip(wild, 0, 6), plan, 6, spatial="hat"))
    with pytest.raises(Exception):
        _sv(bf, u8, rad, plan, 9, spatial="hat")  # the hat takes r_max <= 8


def test_hat_full_size_sampled(bf, oracle):
    H = W = 2048
    img = synth.smooth_field(H, W, noise=5.0, seed=0)
    rad = synth.radius_map(H, W, 8, seed=1)
    plan = bf.Plan(2.0, 20.0, kind="box")
    out = _sv(bf, img, rad, plan, 8, spatial="hat")
    np.testing.assert_array_equal(out, _sv(bf, img, rad, plan, 8, spatial="hat"))
    idx = synth.sample_indices(H, W, 2048, seed=6)
    ref = oracle.bf_brute_sv_at(img, rad, idx, 8, sigma_r=20.0, N=plan.N, spatial="hat")
    err = np.abs(out.ravel()[idx] - ref).max()
    print("space-variant hat 2048^2 max abs err %.3e over %d px" % (err, len(idx)))
    assert err <= TOL


@pytest.mark.parametrize("spatial,r_max", [("box", 8), ("box", 16), ("hat", 8)])
def test_interleaved_channels(bf, oracle, spatial, r_max):
    # H x W x 3 u8, every channel with the same radius map: each channel as
    # the single-channel call (bit for bit) and as the oracle
    import torch
    img = synth.rect_disk_u8(45, 70, C=3, n_shapes=8, seed=4)
    rad = synth.radius_map(45, 70, r_max, seed=7, smooth=False)
    plan = bf.Plan(2.0, 30.0, kind="box")
    t = torch.from_numpy(img).cuda()
    rt = torch.from_numpy(rad).cuda()
    out = bf.forward_space_variant(plan, t, rt, r_max=r_max, spatial=spatial).cpu().numpy()
    assert out.shape == img.shape
    for c in range(3):
        single = _sv(bf, np.ascontiguousarray(img[..., c]), rad, plan, r_max, spatial=spatial)
        np.testing.assert_array_equal(out[..., c], single)
        ref = oracle.bf_brute_sv(img[..., c].astype(np.float64), rad, sigma_r=30.0, r_max=r_max,
                                 N=plan.N, spatial=spatial)
        assert np.abs(out[..., c] - ref).max() <= TOL


def _per_tile_radii(H, W, T, r_max, seed):
    """A radius map whose output tiles (T x T, as the kernel cuts them) each
    have their own largest radius R in [0, r_max]: random radii up to R inside
    the tile, R itself at one corner or edge pixel, so that neighbouring
    tiles build tables of different halos next to each other."""
    rng = np.random.default_rng(seed)
    rad = np.zeros((H, W), np.int32)
    for y0 in range(0, H, T):
        for x0 in range(0, W, T):
            h, w = min(T, H - y0), min(T, W - x0)
            R = int(rng.integers(0, r_max + 1))
            blk = rng.integers(0, R + 1, size=(h, w)).astype(np.int32) if R else np.zeros((h, w), np.int32)
            if rng.random() < 0.5:
                blk[:] = np.minimum(blk, max(R - 1, 0))  # R only at the chosen pixel
            yy, xx = [(0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1), (h // 2, 0)][int(rng.integers(0, 5))]
            blk[yy, xx] = R
            rad[y0:y0 + h, x0:x0 + w] = blk
    return rad


@pytest.mark.parametrize("spatial,r_max,T", [("box", 4, 32), ("box", 8, 32), ("box", 16, 64),
                                             ("hat", 4, 32), ("hat", 8, 32)])
def test_tiles_with_their_own_halos(bf, oracle, spatial, r_max, T):
    # each tile's tables span a halo of its own largest radius: tiles of
    # radius 0 next to tiles of r_max, the largest radius on a tile's corner
    H, W = 2 * T + 23, 3 * T + 9
    img = synth.rectangles(H, W, n_rect=8, noise=10.0, seed=T + r_max)
    rad = _per_tile_radii(H, W, T, r_max, seed=r_max + (7 if spatial == "hat" else 0))
    plan = bf.Plan(3.0, 20.0, kind="box")
    out = _sv(bf, img, rad, plan, r_max, spatial=spatial)
    ref = oracle.bf_brute_sv(img, rad, sigma_r=20.0, r_max=r_max, N=plan.N, spatial=spatial)
    err = np.abs(out - ref).max()
    assert err <= TOL, err
