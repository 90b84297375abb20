"""Failure paths of the training step, made on the host (no GPU fault):

* the dynamic loss scale of a mixed-precision object: a scale so large that
  the scaled 16-bit gradient overflows drops the step (theta, Adam moments
  and the gradient are left as they were, the scale halves, the drop is
  counted), and clean steps double it after the growth interval;
* PRENOM_FLAG_CHECK_FINITE: a NaN target makes the loss non-finite, the call
  reports PRENOM_ERR_NONFINITE and takes no Adam step;
* prenom_autotune: the autotuner's calls and the graph captures happen there,
  leave the object's state unchanged, and none happen in the training loop
  that follows; with PRENOM_FLAG_RETUNE it tunes the step again, likewise.
"""

import numpy as np
import pytest

from helpers import CFG1, case

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


def _dev(rays, obj, **extra):
    import torch

    b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    b["obj"] = obj
    for k, v in extra.items():
        b[k] = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()
    return b


def _object(pkg, precision, seed=71, n_rays=128):
    a, theta, grid, rays, u, cr = case(CFG1, n_rays, 32, 32, seed=seed, hash_range=0.5)
    ctx = pkg.Context(seed=3)
    obj = ctx.create_object(pkg.make_arch(**CFG1, precision=precision), theta)
    ctx.set_prior_grid(obj, grid)
    return ctx, obj, rays, u, cr, grid


def _state(ctx, pkg, obj):
    return [ctx.get_state(obj, w).cpu().numpy() for w in (pkg.PRENOM_STATE_THETA, pkg.PRENOM_STATE_ADAM_M,
                                                          pkg.PRENOM_STATE_ADAM_V, pkg.PRENOM_STATE_GRAD)]


@pytest.mark.parametrize("flags", [0, 8])  # the autotuned (split) form and the fused kernel
def test_fp16_overflow_drops_the_step_and_halves_the_scale(pkg, flags):
    import torch

    ctx, obj, rays, u, cr, _ = _object(pkg, pkg.PRENOM_PRECISION_FP16)
    b = _dev(rays, obj, uniforms=u, c_rand=cr)
    big = float(2 ** 40)  # dL/d(outputs) times 2^40 is far beyond FP16's 65504
    before = _state(ctx, pkg, obj)
    loss = torch.zeros(1, device="cuda")
    ctx.train_step([b], pkg.make_opts(nc=32, nr=32, lr=1e-2, loss_scale_init=big, flags=flags), loss)
    ctx.sync()
    after = _state(ctx, pkg, obj)
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)  # theta, m, v untouched; the gradient cleared (it was zero)
    scale, dropped = ctx.loss_scale(obj)
    assert scale == big / 2 and dropped == 1
    assert np.isfinite(loss.item())  # the loss itself is FP32 and fine
    assert ctx.get_step(obj) == 1  # a dropped step still counts, so the next bias correction moves on
    # with a normal scale the next step trains
    ctx.set_loss_scale(obj, 2.0 ** 15)
    ctx.train_step([b], pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=flags), loss)
    ctx.sync()
    th = ctx.get_state(obj).cpu().numpy()
    assert np.max(np.abs(th - before[0])) > 0
    assert ctx.loss_scale(obj) == (2.0 ** 15, 1)
    ctx.close()


def test_loss_scale_doubles_after_its_growth_interval(pkg):
    import torch

    ctx, obj, rays, u, cr, _ = _object(pkg, pkg.PRENOM_PRECISION_FP16)
    b = _dev(rays, obj, uniforms=u, c_rand=cr)
    ctx.set_loss_scale(obj, 1024.0, growth_interval=3)
    loss = torch.zeros(1, device="cuda")
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-3)
    seen = []
    for _ in range(7):
        ctx.train_step([b], opts, loss)
        seen.append(ctx.loss_scale(obj))
    assert [s for s, _ in seen] == [1024.0, 1024.0, 2048.0, 2048.0, 2048.0, 4096.0, 4096.0]
    assert all(d == 0 for _, d in seen)
    with pytest.raises(pkg.PrenomError):
        ctx.set_loss_scale(obj, 0.5)
    with pytest.raises(pkg.PrenomError):
        ctx.set_loss_scale(obj, 2.0, growth_interval=0)
    o32 = ctx.create_object(pkg.make_arch(**CFG1))
    with pytest.raises(pkg.PrenomError):
        ctx.set_loss_scale(o32, 2.0)
    ctx.close()


@pytest.mark.parametrize("with_loss", [True, False])
def test_check_finite_reports_a_nan_loss_and_skips_adam(pkg, with_loss):
    import torch

    ctx, obj, rays, u, cr, _ = _object(pkg, pkg.PRENOM_PRECISION_FP32)
    bad = dict(rays)
    bad["rgb"] = rays["rgb"].copy()
    obj_rays = np.nonzero(rays["is_obj"])[0]
    bad["rgb"][obj_rays[0], 1] = np.nan  # one object ray with a NaN target colour
    b = _dev(bad, obj, uniforms=u, c_rand=cr)
    before = _state(ctx, pkg, obj)
    loss = torch.zeros(1, device="cuda") if with_loss else None
    with pytest.raises(pkg.PrenomError) as e:
        ctx.train_step([b], pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_CHECK_FINITE), loss)
    assert e.value.code == pkg.PRENOM_ERR_NONFINITE
    ctx.sync()
    after = _state(ctx, pkg, obj)
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)  # no Adam step, the gradient cleared
    assert ctx.get_step(obj) == 0
    if with_loss:
        assert not np.isfinite(loss.item())
    # the same batch without the NaN trains normally under the check
    ctx.train_step([_dev(rays, obj, uniforms=u, c_rand=cr)],
                   pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_CHECK_FINITE), loss)
    assert ctx.get_step(obj) == 1
    ctx.close()


def test_autotune_leaves_the_state_and_the_loop_neither_tunes_nor_captures(pkg):
    import torch

    ctx = pkg.Context(seed=9, stream=torch.cuda.Stream())  # graphs need a stream of its own
    objs, batches = [], []
    for i, prec in enumerate((pkg.PRENOM_PRECISION_FP16, pkg.PRENOM_PRECISION_FP16, pkg.PRENOM_PRECISION_FP32)):
        _, theta, grid, rays, u, cr = case(CFG1, 96 + 64 * i, 32, 32, seed=81 + i, hash_range=0.5)
        o = ctx.create_object(pkg.make_arch(**CFG1, precision=prec), theta)
        ctx.set_prior_grid(o, grid)
        objs.append(o)
        batches.append(_dev(rays, o, uniforms=u, c_rand=cr))
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2)
    before = [_state(ctx, pkg, o) for o in objs]
    ctx.autotune(batches, opts)
    ctx.sync()
    for o, st in zip(objs, before):
        for x, y in zip(st, _state(ctx, pkg, o)):
            np.testing.assert_array_equal(x, y)
        assert ctx.get_step(o) == 0
        if o != objs[-1]:
            assert ctx.loss_scale(o) == (2.0 ** 15, 0)
    report = ctx.tuning_report()
    assert report.count("->") == 2  # the FP16 group and the FP32 group are tuned
    captures, tune_calls = ctx.capture_count()
    assert captures == 2 and tune_calls > 0
    loss = torch.zeros(3, device="cuda")
    for _ in range(6):
        ctx.train_step(batches, opts, loss)
    ctx.sync()
    assert ctx.capture_count() == (captures, tune_calls)
    assert all(ctx.get_step(o) == 6 for o in objs)
    assert np.all(np.isfinite(loss.cpu().numpy()))
    # tuning again on the trained objects: more autotuner calls, the state unchanged,
    # and the loop that follows neither tunes nor captures
    before = [_state(ctx, pkg, o) for o in objs]
    ctx.autotune(batches, pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_RETUNE))
    ctx.sync()
    captures2, tune_calls2 = ctx.capture_count()
    assert tune_calls2 > tune_calls and captures2 >= captures
    for o, st in zip(objs, before):
        for x, y in zip(st, _state(ctx, pkg, o)):
            np.testing.assert_array_equal(x, y)
        assert ctx.get_step(o) == 6
    for _ in range(3):
        ctx.train_step(batches, opts, loss)
    ctx.sync()
    assert ctx.capture_count() == (captures2, tune_calls2)
    assert all(ctx.get_step(o) == 9 for o in objs)
    ctx.close()


def test_timing_report_names_every_group(pkg):
    import torch

    ctx = pkg.Context(seed=4)
    batches = []
    for i, w in enumerate((16, 32)):
        arch = dict(CFG1, width=w)
        _, theta, grid, rays, u, cr = case(arch, 128, 32, 32, seed=91 + i, hash_range=0.5)
        o = ctx.create_object(pkg.make_arch(**arch, precision=pkg.PRENOM_PRECISION_FP16), theta)
        ctx.set_prior_grid(o, grid)
        batches.append(_dev(rays, o, uniforms=u, c_rand=cr))
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_SPLIT)
    ctx.enable_timing(True)
    for _ in range(3):
        ctx.train_step(batches, opts, torch.zeros(2, device="cuda"))
    rep = ctx.timing_report()
    labels = {lab for lab, _, _, _ in rep}
    assert len(labels) == 2 and all("split" in lab for lab in labels)
    assert {k for _, k, _, _ in rep} == {pkg.PRENOM_KERNEL_SAMPLE_ENCODE, pkg.PRENOM_KERNEL_TRAIN,
                                         pkg.PRENOM_KERNEL_SCATTER}
    assert all(n == 3 and ms > 0 for _, _, ms, n in rep)
    ctx.enable_timing(False)
    ctx.close()
