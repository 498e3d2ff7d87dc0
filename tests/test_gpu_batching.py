"""Batching: many functions of uneven bandlimits in one plan, and CUDA-graph
capture of the round trip.

Workload: 256 functions with bandlimits drawn uniformly from {16, 24, ..., 128}
(seeded), TF32x3, complex-normal coefficients; every function's round trip,
and one function of every bandlimit's inverse and forward (of arbitrary,
not band-limited samples) are checked against the FP64 oracle.  The round
trip runs through the plan's own CUDA graphs (sgl_set_graphs) and inside a
caller's graph capture; both must reproduce the direct launches exactly.  The round trip is captured in a
CUDA graph and replayed; replays must reproduce the eager results exactly.
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tolerances import SPLIT_TOL as TF32X3_TOL


@pytest.fixture(scope="module")
def batch():
    from paper_1604_05140_gb300 import Plan
    Bs = inputs.uneven_bandlimits(256)
    plan = Plan.many([int(b) for b in Bs], precision="tf32x3")
    coeffs = [inputs.random_coeffs(int(B), 1, seed=inputs.BASE_SEED + 4 + 10 * k)[0] for k, B in enumerate(Bs)]
    flat = torch.from_numpy(np.concatenate(coeffs)).to(torch.complex64).cuda()
    return plan, Bs, coeffs, flat


def test_uneven_batch_round_trip_and_oracle(batch):
    plan, Bs, coeffs, flat = batch
    s = plan.inverse(flat)
    f = plan.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    checked = set()
    for k, B in enumerate(Bs):
        B = int(B)
        co = plan.coeff_offset(k)
        fk = f[co:co + O.coeff_count(B)]
        err = np.abs(fk - coeffs[k]).max() / np.abs(coeffs[k]).max()
        assert err < TF32X3_TOL, (k, B, err)
        if B not in checked:   # the oracle's inverse of one function of every bandlimit
            so = plan.sample_offset(k)
            sk = s[so:so + 4 * B ** 3].reshape(1, B, 2 * B, 2 * B)
            ref = O.inverse(coeffs[k], B)
            assert np.abs(sk - ref).max() / np.abs(ref).max() < TF32X3_TOL, (k, B)
            checked.add(B)
    assert len(checked) == 15
    plan.check()


def test_uneven_batch_forward_of_arbitrary_samples(batch):
    # the forward transform of samples that are not band-limited (the
    # quadrature of Thm 3.4 of any sample vector): one function of every
    # bandlimit against the oracle's forward of the same samples
    plan, Bs, coeffs, flat = batch
    parts, picked = [], {}
    for k, B in enumerate(Bs):
        B = int(B)
        g = inputs.random_samples(B, 1, seed=inputs.BASE_SEED + 40 + k)[0].astype(np.complex64)
        parts.append(g.reshape(-1))
        if B not in picked:
            picked[B] = (k, g)
    f = plan.forward(torch.from_numpy(np.concatenate(parts)).cuda()).cpu().numpy()
    for B, (k, g) in picked.items():
        co = plan.coeff_offset(k)
        ref = O.forward(g[None], B)[0]
        fk = f[co:co + O.coeff_count(B)]
        assert np.abs(fk - ref).max() / np.abs(ref).max() < TF32X3_TOL, (k, B)
    assert len(picked) == 15
    plan.check()


def test_plan_graphs_match_direct_launches(batch):
    # sgl_set_graphs: the plan captures each call kind and buffer pair once,
    # replays it afterwards, and gives the direct launches' results bit for
    # bit; a caller's own capture still records the plan's launches directly
    plan, Bs, coeffs, flat = batch
    s = torch.empty(plan.sample_shape, dtype=plan.dtype, device="cuda")
    out = torch.empty(plan.coeff_shape, dtype=plan.dtype, device="cuda")
    plan.inverse(flat, out=s)
    plan.forward(s, out=out)
    adj = plan.adjoint(s, of_inverse=True)
    torch.cuda.synchronize()
    eager_s, eager, eager_adj = s.clone(), out.clone(), adj.clone()
    plan.set_graphs(True)
    assert plan.graph_count == 0
    for _ in range(3):
        s.zero_()
        out.zero_()
        plan.inverse(flat, out=s)
        plan.forward(s, out=out)
    torch.cuda.synchronize()
    assert plan.graph_count == 2
    assert torch.equal(s, eager_s) and torch.equal(out, eager)
    out2 = torch.empty_like(out)  # another buffer pair: another graph
    plan.forward(s, out=out2)
    adj2 = torch.empty_like(adj)
    plan.adjoint(s, of_inverse=True, out=adj2)  # another call kind (weights dropped)
    torch.cuda.synchronize()
    assert plan.graph_count == 4
    assert torch.equal(out2, eager) and torch.equal(adj2, eager_adj)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.forward(s, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.forward(s, out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager) and plan.graph_count == 4
    plan.set_graphs(False)
    assert plan.graph_count == 0
    plan.check()


def test_cuda_graph_replay_matches_eager(batch):
    plan, Bs, coeffs, flat = batch
    s = torch.empty(plan.sample_shape, dtype=plan.dtype, device="cuda")
    out = torch.empty(plan.coeff_shape, dtype=plan.dtype, device="cuda")
    plan.inverse(flat, out=s)
    plan.forward(s, out=out)
    torch.cuda.synchronize()
    eager = out.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm the capture stream
        plan.inverse(flat, out=s)
        plan.forward(s, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.inverse(flat, out=s)
        plan.forward(s, out=out)
    out.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    plan.check()
