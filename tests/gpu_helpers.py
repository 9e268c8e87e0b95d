"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and the oracle on
the same seeded scene."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2509_18497_gb300 import api, rgs


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def run_gpu(sc, W=None, alpha_model=rgs.RGS_ALPHA_GAUSS, iterates=False, stats=False, precision=rgs.RGS_FP32,
            checkpoint=0, pairs=False, geometry=False, tensor_cores=-1, mem_budget=0):
    """build -> trace -> solve (-> adjoint with dL/dB = W) on cuda:0; numpy float64 out.
    pairs: the center-to-center transport (the adjoint then also returns dlam);
    tensor_cores: rgs_set_tensor_cores mode of the batched precisions."""
    d = api.upload(sc)
    pipe = api.Pipeline(alpha_model, precision, checkpoint=checkpoint, pairs=pairs, tensor_cores=tensor_cores,
                        mem_budget=mem_budget)
    pipe.build(d)
    pipe.trace(d)
    B, st = pipe.solve(d["E"], d["nb"], stats=stats)
    out = dict(B=B.double().cpu().numpy(), stats=st, pipe=pipe)
    if iterates:
        out["iters"] = [rgs.rgs_get_iterate(pipe.transport, b).double().cpu().numpy() for b in range(d["nb"] + 1)]
    if W is not None:
        g = torch.as_tensor(np.ascontiguousarray(W, np.float32), device="cuda")
        if pairs and geometry:
            dE, dad, dop, dlam, dp, ds, dtu, dtv = pipe.adjoint_pairs_geometry(g)
            out.update(dlam=dlam.double().cpu().numpy(), dp=dp.double().cpu().numpy(), ds=ds.double().cpu().numpy(),
                       dtu=dtu.double().cpu().numpy(), dtv=dtv.double().cpu().numpy())
        elif pairs:
            dE, dad, dop, dlam = pipe.adjoint_pairs(g)
            out["dlam"] = dlam.double().cpu().numpy()
        elif geometry:
            dE, dad, dop, dp, ds, dtu, dtv = pipe.adjoint_geometry(g)
            out.update(dp=dp.double().cpu().numpy(), ds=ds.double().cpu().numpy(),
                       dtu=dtu.double().cpu().numpy(), dtv=dtv.double().cpu().numpy())
        else:
            dE, dad, dop = pipe.adjoint(g)
        out.update(dE=dE.double().cpu().numpy(), dad=dad.double().cpu().numpy(), dop=dop.double().cpu().numpy())
    out["info"] = rgs.rgs_transport_info_get(pipe.transport)
    torch.cuda.synchronize()
    return out


def run_oracle(sc, W=None, alpha_model=O.ALPHA_GAUSS, iterates=False, pairs=False, geometry=False):
    orc = O.Oracle(sc, alpha_model=alpha_model)
    orc = orc.pairs(lam=sc.get("lam")) if pairs else orc.transport()
    out = dict(orc=orc)
    if iterates:
        B, it = orc.solve(E=sc["E"], nb=sc["nb"], iters=True)
        out["iters"] = list(it)
    else:
        B = orc.solve(E=sc["E"], nb=sc["nb"])
    out["B"] = B
    if W is not None:
        out.update(orc.adjoint(W, E=sc["E"], nb=sc["nb"]))
        if geometry:
            out.update(orc.geometry_grad(W, E=sc["E"], nb=sc["nb"]))
    return out
