"""One rank of the template-gradient test (run by test_template_dist.py as a
separate process; gloo on the CPU).  The per-subject term is the oracle's
FP64 LNCC gradient pulled back through the warp adjoint."""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2404_01249_gb300 import synth  # noqa: E402
from paper_2404_01249_gb300.template import template_gradient  # noqa: E402


def oracle_term(template, subject, u, window, cc_eps):
    T, S, U = (t.numpy() for t in (template, subject, u))
    J = oracle.warp(T, U, want_grad=False)
    r = oracle.lncc(S, J, window, cc_eps, want_dJ=True)
    g = oracle.warp_adjoint(r["dJ"], U, T.shape)
    return torch.tensor(r["loss"], dtype=torch.float64), torch.from_numpy(g)


def subjects(shape, idx):
    subs = [torch.from_numpy(synth.voronoi_pair(shape=shape, seed=200 + i)[1].astype(np.float64))
            for i in idx]
    us = [torch.from_numpy(synth.random_field(shape, 2.0, 1.0, seed=300 + i).astype(np.float64))
          for i in idx]
    return subs, us


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    out = sys.argv[1]
    oracle.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shape = (8, 9, 10)
    T = torch.from_numpy(synth.voronoi_pair(shape=shape, seed=199)[0].astype(np.float64))
    per = 2
    subs, us = subjects(shape, range(rank * per, rank * per + per))
    loss, g = template_gradient(T, subs, us, window=3, cc_eps=1e-5, grad_fn=oracle_term)
    np.save(out, np.concatenate([[float(loss)], g.numpy().ravel()]))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
