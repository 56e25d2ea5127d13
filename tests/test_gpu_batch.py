"""Batched lattices (one launch per phase for all members) against stepping
each lattice on its own, and graph replay of batched steps."""
import numpy as np
import pytest

from paper_1710_02375_gb300 import synth

pytestmark = pytest.mark.gpu


def build(inst, coupled, stream, storage=0):
    from paper_1710_02375_gb300.cases import c4_lattice
    return c4_lattice(inst, coupled, stream, storage)


@pytest.mark.parametrize("coupled", [False, True])
def test_batch_matches_individual_steps(coupled):
    import torch
    insts = synth.c4_instances(n=4, seed=3)
    stream = torch.cuda.Stream()
    from paper_1710_02375_gb300.lbm import Batch
    solo = [build(i, coupled, stream) for i in insts]
    for L, _ in solo:
        L.step(150)
    ref = [L.get_populations() for L, _ in solo]
    refb = [b.state()[0] if b else None for _, b in solo]
    group = [build(i, coupled, stream) for i in insts]
    B = Batch([L for L, _ in group])
    B.step(150)
    for k, (L, b) in enumerate(group):
        L.check()
        got = L.get_populations()
        if coupled:
            assert np.max(np.abs(got - ref[k])) <= 1e-9
            assert np.max(np.abs(b.state()[0] - refb[k])) <= 1e-9 * max(1e-12, np.max(np.abs(refb[k])))
        else:
            assert np.array_equal(got, ref[k])
    B.close()


def test_batch_graph_replay_and_autotune():
    import torch
    insts = synth.c4_instances(n=3, seed=11)
    stream = torch.cuda.Stream()
    from paper_1710_02375_gb300.lbm import Batch
    a = [build(i, False, stream) for i in insts]
    b = [build(i, False, stream) for i in insts]
    Ba, Bb = Batch([L for L, _ in a]), Batch([L for L, _ in b])
    Ba.step(40)
    Bb.step_graph(10, 4)
    for (La, _), (Lb, _) in zip(a, b):
        assert np.array_equal(La.get_populations(), Lb.get_populations())
    rows, ctas, us = Ba.autotune(steps=2)
    assert rows in (1, 2, 4, 8) and 3 <= ctas <= 8 and us > 0
    # JSON cache per size bucket: tuned once, then applied without timing
    import json
    import os
    import tempfile
    path = os.path.join(tempfile.mkdtemp(), "tune.json")
    r1, c1, u1 = Ba.autotune(steps=2, cache=path)
    assert u1 is not None and Ba.size_bucket() in json.load(open(path))
    r2, c2, u2 = Bb.autotune(steps=2, cache=path)
    assert (r2, c2, u2) == (r1, c1, None)
