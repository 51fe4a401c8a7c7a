"""One simulation split over several contexts (tpns_options.rank / nranks), all on one GPU:
each context solves its own subdomains and repeats the coarse solve; the sum of the parts of
the glued fields equals the glued fields of the whole simulation.  The contexts are
independent (no context waits for another), so running them on one GPU is the same
computation as running them on separate GPUs."""
import numpy as np
import pytest

import workloads as W
from oracle.scheme import TwoGridOracle
from oracle.scheme3d import TwoGridOracle3D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2311_05170_gb300 import build
    build.build()
    from paper_2311_05170_gb300 import native as N
    return N


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("cfg,prec,nranks", [("small", "fp64", 2), ("small", "fp32", 3), ("graded", "fp32", 2),
                                              ("small3d", "fp32", 3)])
def test_split_parts_sum_to_the_whole(native, cfg, prec, nranks):
    from paper_2311_05170_gb300.shard import reduce_fields
    w = {"small": lambda: W.config_small(nsteps=3), "graded": lambda: W.config_graded(nsteps=3),
         "small3d": lambda: W.config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1, nsteps=3)}[cfg]()
    whole = native.Solver(w, precision=prec)
    whole.step(3)
    ref = whole.fields()
    whole.close()
    parts = []
    for r in range(nranks):
        s = native.Solver(w, precision=prec, rank=r, nranks=nranks)
        s.step(3)
        parts.append(s.fields())
        s.close()
    tot = {k: sum(p[k] for p in parts) for k in ref}
    for k in ref:
        assert rel(tot[k], ref[k]) <= 1e-14, (k, rel(tot[k], ref[k]))
    if cfg in ("small", "small3d"):
        o = TwoGridOracle(w) if cfg == "small" else TwoGridOracle3D(w)
        o.run(3)
        for k in ref:
            assert rel(tot[k], o.fine[k]) <= (1e-10 if prec == "fp64" else 1e-8), k
    # a single process reduces the parts the same way (no collective)
    one = reduce_fields(parts[0], False)
    assert all(np.array_equal(one[k], parts[0][k]) for k in one)
