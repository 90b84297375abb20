"""Training rays from RGB-D keyframes (§III-B "Training Data") on the GPU against
the oracle: the same FP32 geometry in the same operation order, so every
candidate decision, every drawn pixel and every output must be identical."""

import numpy as np
import pytest

import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_01582_gb300 import build

    build.build()
    import paper_2503_01582_gb300 as p

    return p


def _scene(n_kf, H, W, seed, yaw=0.7):
    import synth

    sc = synth.scene_random_csg(seed)
    obj = synth.object_pose([1.0, 2.0, 0.4], yaw, [0.6, 0.5, 0.4])
    kfs = [synth.render_keyframe(sc, p, obj, H, W, 50, 7, depth_noise=0.002, seed=i)
           for i, p in enumerate(synth.keyframe_cameras(n_kf, obj[1], 2.0, seed))]
    # some object pixels lose their depth (invalid readings drop those rays)
    rng = np.random.default_rng(seed)
    for k in kfs:
        k["depth"][rng.random(k["depth"].shape) < 0.05] = 0.0
    state = dict(instance=7, R_wo=obj[0], centre=obj[1], size=obj[2])
    return sc, kfs, state


def _dev_kf(k):
    import torch

    return dict(k, rgb=torch.from_numpy(k["rgb"]).cuda(), depth=torch.from_numpy(k["depth"]).cuda(),
                mask=torch.from_numpy(k["mask"]).cuda())


@pytest.mark.parametrize("n_kf,H,W,n_rays", [(1, 48, 64, 500), (3, 120, 160, 4096), (8, 480, 640, 20000)])
def test_make_rays_bit_exact_against_oracle(pkg, n_kf, H, W, n_rays):
    import torch

    sc, kfs, state = _scene(n_kf, H, W, seed=n_kf)
    draws = np.random.default_rng(1).integers(0, 2 ** 32, n_rays, dtype=np.uint64).astype(np.uint32)
    want, n_want = orc.make_rays(kfs, state, draws)
    ctx = pkg.Context(seed=5)
    got, n_got = ctx.make_rays([_dev_kf(k) for k in kfs], state, n_rays,
                               draws=torch.from_numpy(draws.view(np.int32)).cuda(), count=True)
    assert n_got == n_want > 0
    for k in ("o", "d", "rgb", "depth", "is_obj"):
        np.testing.assert_array_equal(got[k].cpu().numpy(), want[k], err_msg=k)
    ctx.close()


def test_make_rays_internal_philox_and_training(pkg):
    """Without draws the words come from Philox4x32-10 keyed as documented; the
    batch trains an object directly (the loss falls)."""
    import torch
    from helpers import CFG1
    from synth import prior_grid

    sc, kfs, state = _scene(4, 120, 160, seed=9)
    n = 2048
    call0 = [orc.philox4x32_10([j >> 2, 0, 0, 0x52415953], [5, 0])[j & 3] for j in range(n)]
    want, _ = orc.make_rays(kfs, state, np.array(call0, np.uint32))
    ctx = pkg.Context(seed=5)
    dkf = [_dev_kf(k) for k in kfs]
    got = ctx.make_rays(dkf, state, n)
    for k in ("o", "d", "depth", "is_obj"):
        np.testing.assert_array_equal(got[k].cpu().numpy(), want[k], err_msg=k)
    # the second call draws with call = 1
    call1 = [orc.philox4x32_10([j >> 2, 0, 1, 0x52415953], [5, 0])[j & 3] for j in range(n)]
    want1, _ = orc.make_rays(kfs, state, np.array(call1, np.uint32))
    got1 = ctx.make_rays(dkf, state, n)
    np.testing.assert_array_equal(got1["o"].cpu().numpy(), want1["o"])
    a = CFG1
    obj = ctx.create_object(pkg.make_arch(L=a["L"], F=a["F"], log2T=a["log2T"], n_min=a["n_min"], n_max=a["n_max"],
                                          width=a["width"], hidden=a["hidden"]))
    ctx.set_prior_grid(obj, prior_grid(sc, 32, 0))
    loss = torch.zeros(1, device="cuda")
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2)
    hist = []
    for step in range(60):
        b = ctx.make_rays(dkf, state, 512)
        b["obj"] = obj
        ctx.train_step([b], opts, loss)
        hist.append(loss.item())
    assert np.all(np.isfinite(hist)) and np.mean(hist[-10:]) < 0.7 * np.mean(hist[:3]), hist
    ctx.close()
