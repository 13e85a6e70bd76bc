"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np

import oracle as O


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def to_dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make_gpu(p: O.Problem, vcycle_fp32=False, **kw):
    import paper_1401_7824_gb300 as G
    torch_cuda()
    return G.Isdc(p.ndim, p.n, p.nu, p.M, p.dt, smoother=p.smoother, nu1=p.nu1, nu2=p.nu2,
                  omega=p.omega, vcycle_fp32=vcycle_fp32,
                  reaction=G.ISDC_REACTION_ALLEN_CAHN if p.reaction == O.REACTION_ALLEN_CAHN
                  else G.ISDC_REACTION_NONE,
                  tol=p.tol, max_sweeps=p.max_sweeps, mg_tol=p.mg_tol, mg_max_cycles=p.mg_max_cycles,
                  nodes={O.NODES_LOBATTO: G.ISDC_NODES_GAUSS_LOBATTO, O.NODES_RADAU_RIGHT: G.ISDC_NODES_RADAU_RIGHT,
                         O.NODES_LEGENDRE: G.ISDC_NODES_GAUSS_LEGENDRE}[p.nodes],
                  stencil={O.STENCIL_SECOND_ORDER: G.ISDC_STENCIL_SECOND_ORDER,
                           O.STENCIL_COMPACT: G.ISDC_STENCIL_COMPACT}[p.stencil],
                  equation={O.EQUATION_REACTION_DIFFUSION: G.ISDC_EQUATION_REACTION_DIFFUSION,
                            O.EQUATION_BURGERS: G.ISDC_EQUATION_BURGERS}[p.equation], **kw)
