"""Batching: many functions of uneven bandlimits in one plan, and CUDA-graph
capture of the round trip.

Workload: 256 functions with bandlimits drawn uniformly from {16, 24, ..., 128}
(seeded), TF32x3, complex-normal coefficients; every function's round trip,
and one function of every bandlimit's inverse and forward (of arbitrary,
not band-limited samples) are checked against the FP64 oracle.  The round trip is captured in a
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
