"""The allocation-free training step against the regular one.

prenom_train_step_noalloc() serves callers that cannot allocate device memory
while they train (a mapping front end that reserved the GPU's memory budget up
front, a host framework whose allocator owns the device pool, a real-time
thread that cannot take cudaMalloc's implicit synchronisation).  It keeps its
gradient accumulator in a fixed array inside the library, so this test calls
it twice in a row through the C ABI -- the second call must not see the
first call's gradients -- and compares loss, Adam moments and parameters with
prenom_train_step() on an identical object after each call.  Around the
second call the device's free memory and torch's reserved pool must not move.
"""

import numpy as np
import pytest

from helpers import CFG1, case, rel

import oracle as orc

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4


def test_noalloc_step_matches_train_step_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_01582_gb300 import build

    build.build()
    import paper_2503_01582_gb300 as pkg
    from paper_2503_01582_gb300 import _abi, ray_batch

    a, theta, grid, rays, u, cr = case(CFG1, 192, 32, 32, seed=61, hash_range=0.5)
    arch = pkg.make_arch(**{k: v for k, v in CFG1.items()})
    n = orc.param_count(a)
    assert n <= _abi.PRENOM_NOALLOC_MAX_PARAMS
    lr = 1e-2
    opts = pkg.make_opts(nc=32, nr=32, lr=lr)

    # regular path: a library-owned object
    ctx = pkg.Context(seed=5)
    obj = ctx.create_object(arch, theta)
    ctx.set_prior_grid(obj, grid)

    # allocation-free path: caller-owned theta, Adam moments, grid and loss
    th = torch.from_numpy(theta).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    g_dev = torch.from_numpy(grid).cuda()
    loss_a = torch.zeros(1, device="cuda")
    loss_b = torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()

    half = {k: [x[:96], x[96:]] for k, x in rays.items()}
    for call in range(2):
        b = {k: torch.from_numpy(np.ascontiguousarray(half[k][call])).cuda() for k in half}
        b["obj"] = obj
        b["uniforms"] = torch.from_numpy(np.ascontiguousarray(u[96 * call:96 * (call + 1)])).cuda()
        b["c_rand"] = torch.from_numpy(np.ascontiguousarray(cr[96 * call:96 * (call + 1)])).cuda()
        # reference gradient of this call, for telling Adam's sign-sensitive entries apart
        ref = pkg.Context(seed=5)
        robj = ref.create_object(arch, ctx.get_state(obj))
        ref.set_prior_grid(robj, grid)
        ref.set_step(robj, call)
        ref.train_step([dict(b, obj=robj)], pkg.make_opts(nc=32, nr=32, flags=pkg.PRENOM_FLAG_NO_ADAM))
        g_ref = ref.get_state(robj, pkg.PRENOM_STATE_GRAD).cpu().numpy()
        ref.close()

        ctx.train_step([b], opts, loss_a)
        rb = ray_batch(b)
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        _abi.prenom_train_step_noalloc(arch, th.data_ptr(), m.data_ptr(), v.data_ptr(), call, g_dev.data_ptr(),
                                       grid.shape[0], rb, opts, loss_b.data_ptr(), stream.cuda_stream, 5)
        torch.cuda.synchronize()
        if call == 1:  # past the first call's one-time set-up: no device memory is taken
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0

        assert abs(loss_b.item() - loss_a.item()) <= FWD_TOL * abs(loss_a.item())
        ma = ctx.get_state(obj, pkg.PRENOM_STATE_ADAM_M).cpu().numpy()
        va = ctx.get_state(obj, pkg.PRENOM_STATE_ADAM_V).cpu().numpy()
        ta = ctx.get_state(obj, pkg.PRENOM_STATE_THETA).cpu().numpy()
        assert rel(m.cpu().numpy(), ma) <= GRAD_TOL
        assert rel(v.cpu().numpy(), va) <= GRAD_TOL
        # Adam divides by |g|: entries whose gradient is at the rounding floor may
        # step either way, the rest must agree
        sure = np.abs(g_ref) > 1e-5 * np.abs(g_ref).max()
        d = np.abs(th.cpu().numpy() - ta)
        assert np.max(d[sure]) <= GRAD_TOL * np.abs(ta).max()
        assert np.max(d, initial=0.0) <= 2.01 * lr * (call + 1)

    # objects beyond the fixed array are refused with a clear error
    big = pkg.make_arch(L=16, log2T=19, n_min=16, n_max=2048, width=64, hidden=2)
    with pytest.raises(_abi.PrenomError) as e:
        _abi.prenom_train_step_noalloc(big, th.data_ptr(), m.data_ptr(), v.data_ptr(), 0, g_dev.data_ptr(),
                                       grid.shape[0], ray_batch(b), opts, 0, stream.cuda_stream, 5)
    assert e.value.code == _abi.PRENOM_ERR_INVALID_ARG
    assert "at most" in _abi.prenom_last_error(None)
    ctx.close()
