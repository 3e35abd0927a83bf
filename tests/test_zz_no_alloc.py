"""dses_vote_static: the rotation vote for callers that cannot allocate.

Real-time loops replayed from captured CUDA graphs, hosts that reserve all
device memory up front and plugins whose host application owns the allocator
cannot call cudaMalloc while they run. dses_vote_static keeps its scratch in a
static device array instead; this checks, through the C ABI, that two calls in
a row give the per-rotation translation modes (k*, V) of the allocating path,
for 32-bit counters in one slab, 16-bit counters in x-slabs, and boxes with an
even extent (the entry point's generic rounding path, which the allocating
path never takes: it pads every extent to an odd one), and that sizes beyond
the static scratch are refused. Integer outputs: bit-exact, except where the
two paths' FP32 roundings may put a pair on either side of a voxel face, which
the FP64 oracle must then confirm (a boundary pair within 1e-5). It lives in a
file pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_vote(torch, capi, X, Y, R, params, n):
    dev = torch.device("cuda", 0)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).to(dev)
    Rd = torch.from_numpy(np.ascontiguousarray(R.reshape(-1, 9))).to(dev)
    out = torch.empty((n, 4), dtype=torch.int32, device=dev)
    got = []
    for _ in range(2):  # two calls in a row share the static scratch
        out.fill_(-7)
        torch.cuda.synchronize()
        st = capi.dses_vote_static(0, 0, Xd.data_ptr(), len(X), Yd.data_ptr(), len(Y), Rd.data_ptr(), n, params,
                                   out.data_ptr())
        assert st == capi.DSES_OK
        torch.cuda.synchronize()
        got.append(out.cpu().numpy())
    return got, (Xd, Rd, out)


def _compare(got, k_ref, V_ref, X, Y, R64, params):
    """(k*, V) equal to the allocating path's, else both confirmed by the oracle."""
    import oracle

    f32 = lambda v: float(np.float32(v))
    delta = f32(params.delta_t if params.delta_t > 0 else params.epsilon)
    lo, hi = oracle.lattice_box([f32(v) for v in params.t_center], [f32(v) for v in params.t_half], delta)
    differ = 0
    for g in got:
        same = np.all(g[:, :3] == k_ref, axis=1) & (g[:, 3].astype(np.uint32) == V_ref)
        for r in np.nonzero(~same)[0]:
            differ += 1
            for k, V in ((g[r, :3], int(g[r, 3])), (k_ref[r], int(V_ref[r]))):
                assert oracle.vote_consistent(X, Y, R64[r], delta, lo, hi, np.asarray(k), V) > 0, r
    return differ


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
    got, (X, Rd, out) = _static_vote(torch, capi, p.X, p.Y, R, params, n)
    for g in got:
        assert np.array_equal(g[:, :3], k_ref)
        assert np.array_equal(g[:, 3].astype(np.uint32), V_ref)
    big = torch.zeros((8193, 3), dtype=torch.float32, device=X.device)
    st = capi.dses_vote_static(0, 0, X.data_ptr(), len(p.X), big.data_ptr(), 8193, Rd.data_ptr(), n, params,
                               out.data_ptr())
    assert st == capi.DSES_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["u16_even_x_slabs", "u16_even_y", "u32_even_z"])
def test_static_vote_other_layouts(case):
    torch = pytest.importorskip("torch")
    import oracle
    from paper_2502_00115_b300 import build, capi, synth

    build.build()
    if case.startswith("u16"):
        # 128 x 256 points (N M <= 65535: 16-bit counters), a 90 x 91 x 91 or
        # 91 x 90 x 91 box: x-slabs of 11 planes, the last one of 2 (even)
        p = synth.tiny_problem(5, hopf_n=2)
        centre = (0.01, 0.0, 0.0) if case == "u16_even_x_slabs" else (0.0, 0.01, 0.0)
        params = capi.make_params(metric="trunc_l1", epsilon=p.epsilon, tau=p.tau, t_center=centre,
                                  t_half=p.t_half)
        hopf_n = 2
    else:
        # 32-bit counters in one slab, a 21 x 21 x 20 box off the lattice centre
        p = synth.modelnet_like_problem(7, m=900, keep=0.6, hopf_n=2)
        params = capi.make_params(metric="trunc_l1", epsilon=p.epsilon, tau=p.tau, t_center=(0.0, 0.0, 0.02),
                                  t_half=(0.4, 0.4, 0.4))
        hopf_n = 2
    n = 72 * hopf_n**3
    with capi.Context(0) as ctx:
        t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
        k_ref, V_ref, _, _, _ = ctx.debug(ctx.problem(t, p.X, capi.hopf_grid(hopf_n), params), n)
        R = ctx.rotation_grid(capi.hopf_grid(hopf_n))
    got, _ = _static_vote(torch, capi, p.X, p.Y, R, params, n)
    differ = _compare(got, k_ref, V_ref, p.X, p.Y, R.astype(np.float64), params)
    assert differ <= 0.02 * n * len(got), differ
    # and the oracle's own mode on a sample of rotations (its FP64 decisions at
    # the FP32 rotations, so only boundary pairs may differ)
    f32 = lambda v: float(np.float32(v))
    P = oracle.make_params(metric="trunc_l1", epsilon=f32(params.epsilon), t_center=[f32(v) for v in params.t_center],
                           t_half=[f32(v) for v in params.t_half])
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    for r in np.random.default_rng(0).choice(n, size=40, replace=False):
        k_o, V_o, _, _, _ = oracle.eval_rotation(p.X, p.Y, R[r].astype(np.float64), P)
        g = got[1][r]
        if not (np.array_equal(g[:3], k_o) and int(g[3]) == V_o):
            assert oracle.vote_consistent(p.X, p.Y, R[r].astype(np.float64), P.delta_t, lo, hi, g[:3],
                                          int(g[3])) > 0, r
