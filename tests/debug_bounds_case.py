"""One small workload run twice by tests/test_gpu_debug_bounds.py: with the
regular library in the test process and with the bounds-checked debug build
(PRENOM_DEBUG_BOUNDS=1) in a child process.  It samples from uniforms (prior
lookups), runs the fused FP32 kernel, the split FP16 form (sampling-encoding,
tensor-core and scatter kernels), a batched step of three objects with Adam and
a render, and returns every output for comparison.

Run as a script it writes the outputs of the library it loads to an .npz file."""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
for p in (HERE, os.path.dirname(HERE)):
    if p not in sys.path:
        sys.path.insert(0, p)

from helpers import CFG1, case  # noqa: E402

N_RAYS, NR, NC = 128, 32, 32


def _batch(rays, u, cr, obj):
    import torch

    b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    b["uniforms"] = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    b["c_rand"] = torch.from_numpy(np.ascontiguousarray(cr)).cuda()
    b["obj"] = obj
    return b


def run(pkg) -> dict:
    import torch

    specs = [(dict(CFG1), 0, 11), (dict(CFG1), 1, 12), (dict(CFG1, width=16, hidden=1, log2T=12), 0, 13)]
    ctx = pkg.Context(seed=3)
    ids, batches = [], []
    for arch, prec, seed in specs:
        _, theta, grid, rays, u, cr = case(arch, N_RAYS, NR, NC, seed=seed, hash_range=0.5)
        oid = ctx.create_object(pkg.make_arch(L=arch["L"], log2T=arch["log2T"], n_min=16, n_max=arch["n_max"],
                                              width=arch["width"], hidden=arch["hidden"], lambda_d=0.1,
                                              precision=prec), theta)
        ctx.set_prior_grid(oid, grid)
        ids.append(oid)
        batches.append(_batch(rays, u, cr, oid))
    out = {}
    loss = torch.zeros(len(ids), device="cuda")
    # one object at a time: the fused FP32 kernel, then the split FP16 form
    for k, flags in ((0, pkg.PRENOM_FLAG_FUSED), (1, pkg.PRENOM_FLAG_SPLIT)):
        opts = pkg.make_opts(nc=NC, nr=NR, flags=flags | pkg.PRENOM_FLAG_NO_ADAM)
        ctx.train_step([batches[k]], opts, loss[k:k + 1])
        out[f"grad{k}"] = ctx.get_state(ids[k], pkg.PRENOM_STATE_GRAD).cpu().numpy()
        ctx.zero_grads(ids[k])
    # a batched step of the three objects (untuned split form) with Adam
    ctx.train_step(batches, pkg.make_opts(nc=NC, nr=NR, lr=1e-2, flags=pkg.PRENOM_FLAG_SPLIT), loss)
    out["loss"] = loss.cpu().numpy()
    for k, oid in enumerate(ids):
        out[f"theta{k}"] = ctx.get_state(oid).cpu().numpy()
    r = ctx.render(batches[0], pkg.make_opts(nc=NC, nr=NR), want_samples=True)
    for key in ("rgb", "depth", "acc", "bins", "t"):
        out["render_" + key] = r[key].cpu().numpy()
    ctx.sync()  # raises on a nonzero device status (PRENOM_ERR_DEVICE_BOUNDS in the debug build)
    ctx.close()
    return out


if __name__ == "__main__":
    import torch

    torch.cuda.set_device(0)
    from paper_2503_01582_gb300 import build

    build.build(debug_bounds=os.environ.get("PRENOM_DEBUG_BOUNDS") == "1")
    import paper_2503_01582_gb300 as pkg

    np.savez(sys.argv[1], **run(pkg))
