"""GPU parity of ff_project_sprites (soft sprites, paper Appendix A) against the oracle.

The oracle is fed the GPU's own states, which isolates the render step from the
integration.  Coverage (q < 1) is decided in FP32 on both sides with the same
roundings, so pixels the oracle leaves untouched must stay exactly 0.  The
values are FP32 sums in an unspecified order: each pixel channel must lie within
(n + 8) * 2^-24 * sum|c_i| of the FP64 sum, n being its number of fragments
(the first-order bound of any ordering of n FP32 additions, plus the rounding
of each contribution).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300.workloads import LORENZ_PARAMS, look_at_perspective, workload  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -24
COLOURS = [[1.0, 0.25, 0.0, 1.0], [0.0, 0.5, 1.0, -0.75], [0.3, -1.0, 0.6, 2.0]]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def stream():
    return torch.cuda.current_stream().cuda_stream


def lorenz_system(counts, box=([-30, -30, 0], [30, 30, 60]), seeds=(11, 12, 13)):
    s = ff.System("lorenz", LORENZ_PARAMS, sum(counts), stream=stream())
    for c, sd in zip(counts, seeds):
        s.seed(c, box[0], box[1], 1, sd)
    return s


def state_of(s):
    n, _, dim, _ = s.info()
    x = np.empty((dim, n), np.float32)
    s.get_state(x)
    return x


def groups_of(counts):
    return np.concatenate([np.full(c, g, np.int32) for g, c in enumerate(counts)])


def gpu_sprites(s, view, sprite, W, H, prefill=None):
    img = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    if prefill is not None:
        img.copy_(torch.from_numpy(prefill))
    s.project_sprites(view, sprite, img)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64)


def check(got, want, absum, frags, prefill=None):
    base = np.zeros_like(want) if prefill is None else prefill.astype(np.float64)
    bound = (frags[:, :, None] + 8.0) * U * (absum + np.abs(base))
    err = np.abs(got - (want + base))
    assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())
    untouched = frags == 0
    np.testing.assert_array_equal(got[untouched], base[untouched])


TECHNIQUES = [ff.FF_SPRITE_DIRECT, ff.FF_SPRITE_TILED]


@pytest.mark.parametrize("technique", TECHNIQUES)
@pytest.mark.parametrize("radius", [0.75, 1.5, 4.0, 32.0])
def test_2d_sprites_match_oracle(radius, technique):
    counts = [2003, 1500, 1500]  # ragged: 5003 particles
    s = lorenz_system(counts)
    s.step(150, 0.001)
    W, H = 160, 96
    lo, hi = (-25.0, 2.0), (25.0, 55.0)  # particles spill over every edge of the window
    view = dict(ndim_view=2, axes=(0, 2), lo=lo, hi=hi, width=W, height=H)
    sprite = ff.make_sprite(radius, 0.8, COLOURS, technique)
    got = gpu_sprites(s, view, sprite, W, H)
    x = state_of(s)
    want, absum, frags = oracle.sprites2d(x[0], x[2], lo, hi, W, H, radius, 0.8, COLOURS, group=groups_of(counts))
    assert frags.sum() > 0
    check(got, want, absum, frags)


@pytest.mark.parametrize("technique", TECHNIQUES)
def test_3d_perspective_masked_and_accumulated(technique):
    counts = [1000, 777, 1201]
    s = lorenz_system(counts)
    s.step(300, 0.001)
    W, H = 128, 80
    # camera at (60, 60, 80) looking at (0, 0, 25), 45 degree field of view
    mvp = look_at_perspective((60.0, 60.0, 80.0), (0.0, 0.0, 25.0), (0.0, 0.0, 1.0), 45.0, W / H, 1.0, 500.0)
    view = dict(ndim_view=3, axes=(0, 1, 2), mvp=mvp, width=W, height=H, group_mask=0b101, accumulate=1)
    rng = np.random.default_rng(4)
    prefill = rng.uniform(-1, 1, (H, W, 4)).astype(np.float32)
    sprite = ff.make_sprite(2.5, 1.3, COLOURS, technique)
    got = gpu_sprites(s, view, sprite, W, H, prefill=prefill)
    x = state_of(s)
    g = groups_of(counts)
    want, absum, frags = oracle.sprites3d(x[0], x[1], x[2], np.asarray(mvp, np.float32), W, H, 2.5, 1.3, COLOURS,
                                          group=g, include=(g != 1))
    assert frags.sum() > 0
    check(got, want, absum, frags, prefill=prefill)


@pytest.mark.parametrize("technique", TECHNIQUES)
def test_host_image_and_parameter_axis(technique):
    # bifurcation view: per-particle r on the x axis, z on y; host image, cleared by the call
    s = ff.System("lorenz", LORENZ_PARAMS, 4099, stream=stream())
    s.seed(4099, [-20, -20, 0], [20, 20, 40], 1, 21)
    s.set_particle_param(1, 0.0, 50.0)
    s.step(400, 0.001)
    W, H = 200, 100
    view = dict(ndim_view=2, axes=(3, 2), lo=(0.0, 0.0), hi=(50.0, 80.0), width=W, height=H)
    img = np.full((H, W, 4), 7.0, np.float32)  # stale content: accumulate = 0 clears it
    s.project_sprites(view, ff.make_sprite(1.25, 1.0, COLOURS, technique), img)
    x = state_of(s)
    r = np.empty(4099, np.float32)
    s.get_particle_param(r)
    want, absum, frags = oracle.sprites2d(r, x[2], (0.0, 0.0), (50.0, 80.0), W, H, 1.25, 1.0, COLOURS)
    check(img.astype(np.float64), want, absum, frags)


@pytest.mark.parametrize("technique", TECHNIQUES + [ff.FF_SPRITE_AUTO])
def test_full_size_lorenz_frame(technique):
    # the lorenz_4M workload (4,194,304 particles, 75% forward / 25% backward) after 2 frames,
    # x-z view into 1920 x 1080, forward and backward groups in different colours
    w = workload("lorenz_4M")
    s = ff.System("lorenz", w["params"], sum(g["count"] for g in w["groups"]), stream=stream())
    for g in w["groups"]:
        s.seed(g["count"], g["lo"], g["hi"], g["direction"], g["seed"])
    s.step(400, w["dt"])
    v = w["view"]
    W, H = v["width"], v["height"]
    view = dict(ndim_view=2, axes=tuple(v["axes"]), lo=tuple(v["lo"]), hi=tuple(v["hi"]), width=W, height=H)
    cols = [[1.0, 0.6, 0.2, 1.0], [0.2, 0.4, 1.0, 1.0]]
    got = gpu_sprites(s, view, ff.make_sprite(1.5, 0.05, cols, technique), W, H)
    x = state_of(s)
    counts = [g["count"] for g in w["groups"]]
    ax = v["axes"]
    want, absum, frags = oracle.sprites2d(x[ax[0]], x[ax[1]], v["lo"], v["hi"], W, H, 1.5, 0.05, cols,
                                          group=groups_of(counts))
    assert frags.max() > 100  # dense pixels: the summation-order bound is exercised
    check(got, want, absum, frags)


@pytest.mark.parametrize("technique", TECHNIQUES)
def test_empty_and_masked_out(technique):
    s = ff.System("lorenz", LORENZ_PARAMS, 64, stream=stream())
    W, H = 32, 16
    view = dict(ndim_view=2, axes=(0, 2), lo=(-30.0, 0.0), hi=(30.0, 60.0), width=W, height=H)
    img = torch.full((H, W, 4), 3.0, device="cuda")
    s.project_sprites(view, ff.make_sprite(2.0, technique=technique), img)  # no particles: only cleared
    assert float(img.abs().max()) == 0.0
    s.seed(64, [-30, -30, 0], [30, 30, 60], 1, 1)
    img.fill_(3.0)
    s.project_sprites(dict(view, group_mask=0), ff.make_sprite(2.0, technique=technique), img)
    assert float(img.abs().max()) == 0.0


def test_argument_errors():
    s = lorenz_system([64])
    W, H = 32, 16
    view = dict(ndim_view=2, axes=(0, 2), lo=(-30.0, 0.0), hi=(30.0, 60.0), width=W, height=H)
    img = torch.zeros((H * W * 4 + 4,), device="cuda")
    for sp in (ff.make_sprite(0.0), ff.make_sprite(33.0), ff.make_sprite(float("nan")),
               ff.make_sprite(1.0, float("inf")), ff.make_sprite(1.0, 1.0, [[float("nan"), 0, 0, 0]])):
        with pytest.raises(ff.FFError) as e:
            s.project_sprites(view, sp, img)
        assert e.value.status == ff.FF_ERR_INVALID_ARG
    with pytest.raises(ff.FFError) as e:  # device image not 16-byte aligned: rejected on the host
        s.project_sprites(view, ff.make_sprite(1.0), img.data_ptr() + 4)
    assert e.value.status == ff.FF_ERR_INVALID_ARG
    with pytest.raises(ff.FFError) as e:
        s.project_sprites(view, ff.make_sprite(1.0, technique=3), img)
    assert e.value.status == ff.FF_ERR_INVALID_ARG
    big = dict(view, width=4096, height=4096)  # 16,384 tiles: more than the tiled technique takes
    small = torch.zeros(4, device="cuda")
    with pytest.raises(ff.FFError) as e:  # raw pointer: the library itself rejects the view
        s.project_sprites(big, ff.make_sprite(1.0, technique=ff.FF_SPRITE_TILED), small.data_ptr())
    assert e.value.status == ff.FF_ERR_UNSUPPORTED
