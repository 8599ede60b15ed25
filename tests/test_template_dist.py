"""Template gradient across ranks (gloo, world size 2, CPU): every rank gets
the mean over all ranks' subjects, equal to the single-process mean."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2404_01249_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_template_gradient_allreduce_two_ranks(tmp_path, orc):
    import dist_template_worker as w
    from paper_2404_01249_gb300.template import template_gradient
    port = free_port()
    procs, outs = [], []
    for rank in range(2):
        out = str(tmp_path / f"rank{rank}.npy")
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "dist_template_worker.py"),
                                       out], env=env))
        outs.append(out)
    for p in procs:
        assert p.wait(timeout=300) == 0
    shape = (8, 9, 10)
    T = torch.from_numpy(synth.voronoi_pair(shape=shape, seed=199)[0].astype(np.float64))
    subs, us = w.subjects(shape, range(4))
    loss, g = template_gradient(T, subs, us, window=3, cc_eps=1e-5, grad_fn=w.oracle_term)
    ref = np.concatenate([[float(loss)], g.numpy().ravel()])
    for out in outs:
        got = np.load(out)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)


def test_template_gradient_argument_checks():
    from paper_2404_01249_gb300.template import template_gradient
    T = torch.zeros(2, 2, 2, dtype=torch.float64)
    with pytest.raises(ValueError):
        template_gradient(T, [T], [], grad_fn=lambda *a: (0.0, T))
    with pytest.raises(ValueError):
        template_gradient(T, [], [], grad_fn=lambda *a: (0.0, T))
