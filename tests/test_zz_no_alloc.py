"""dses_vote_static: the rotation vote for callers that cannot allocate.

Real-time loops replayed from captured CUDA graphs, hosts that reserve all
device memory up front and plugins whose host application owns the allocator
cannot call cudaMalloc while they run. dses_vote_static keeps its scratch in a
static device array instead; this checks, through the C ABI, that two calls in
a row give exactly the per-rotation translation modes (k*, V) of the
allocating path (integer outputs: bit-exact), and that sizes beyond the static
scratch are refused. It lives in a file pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_vote_matches_allocating_path_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2502_00115_b300 import build, capi, synth

    build.build()
    p = synth.modelnet_like_problem(3, m=1000, keep=0.7, hopf_n=3)
    n = 72 * 27
    params = capi.make_params(metric=p.metric, epsilon=p.epsilon, tau=p.tau, t_half=p.t_half)
    with capi.Context(0) as ctx:
        t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
        k_ref, V_ref, _, _, _ = ctx.debug(ctx.problem(t, p.X, capi.hopf_grid(3), params), n)
        R = ctx.rotation_grid(capi.hopf_grid(3))
    dev = torch.device("cuda", 0)
    X = torch.from_numpy(p.X).to(dev)
    Y = torch.from_numpy(p.Y).to(dev)
    Rd = torch.from_numpy(np.ascontiguousarray(R.reshape(-1, 9))).to(dev)
    out = torch.empty((n, 4), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    for _ in range(2):
        out.fill_(-7)
        torch.cuda.synchronize()
        st = capi.dses_vote_static(0, 0, X.data_ptr(), len(p.X), Y.data_ptr(), len(p.Y), Rd.data_ptr(), n, params,
                                   out.data_ptr())
        assert st == capi.DSES_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got[:, :3], k_ref)
        assert np.array_equal(got[:, 3].astype(np.uint32), V_ref)
    big = torch.zeros((8193, 3), dtype=torch.float32, device=dev)
    st = capi.dses_vote_static(0, 0, X.data_ptr(), len(p.X), big.data_ptr(), 8193, Rd.data_ptr(), n, params,
                               out.data_ptr())
    assert st == capi.DSES_ERR_INVALID_ARG
