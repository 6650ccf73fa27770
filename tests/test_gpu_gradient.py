"""GPU adjoint (st_backward) against the oracle's float64 analytic gradient (the emitter gradient
including the specular paths through their hit points), and the autograd
wrapper against st_backward, on frozen path sets.  Bar: relative error <= 1e-3 per gradient block
(the oracle's gradient is itself pinned to float64 central differences in test_oracle_spectra)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-3


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def torch_st():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    return torch, st


def grads_vs_oracle(torch, st, wl, curv=None, mode=0):
    import oracle
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl, None if curv is None else st.curv_params(sample_budget=curv))
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, reflection_mode=mode)
    S = ctx.simulate(sc, p)
    rng = np.random.default_rng(7)
    target = torch.as_tensor(rng.normal(size=S.shape) + 1j * rng.normal(size=S.shape), dtype=torch.complex64,
                             device=S.device) * S.abs().mean()
    G = 2.0 * (S - target)
    gk, gm, ge = ctx.backward(sc, G, wl.k_band.shape[0], wl.k_band.shape[1])
    o = oracle.simulate(wl, curv=None if curv is None else dict(budget=curv), reflection_mode=mode)
    dk, dmic, demit = oracle.spectra_grad(o["params"], o["rec"], wl.dirs, wl.tri_mat, G.cpu().numpy().astype(np.complex128),
                                          o.get("cand_tri"), o.get("cand_p"), o.get("cand_keep"), o["direct_vis"],
                                          tri_nrm=oracle.tri_normals(wl.verts, wl.tris))
    return gk.cpu().numpy(), gm.cpu().numpy(), ge.cpu().numpy(), dk, dmic, demit


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_workload_matches_oracle(torch_st, mode):
    torch, st = torch_st
    wl = synth.gradient_problem(n_rays=2000)
    wl.n_bins = 64
    gk, gm, ge, dk, dmic, demit = grads_vs_oracle(torch, st, wl, mode=mode)
    assert rel(gk, dk) <= TOL, rel(gk, dk)
    assert rel(gm, dmic) <= TOL, rel(gm, dmic)
    assert rel(ge, demit) <= TOL, rel(ge, demit)


def test_clutter_gradient_with_diffraction(torch_st):
    torch, st = torch_st
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=6, n_bins=40)
    gk, gm, ge, dk, dmic, demit = grads_vs_oracle(torch, st, wl, curv=100_000)
    assert rel(gk, dk) <= TOL, rel(gk, dk)
    assert rel(gm, dmic) <= TOL, rel(gm, dmic)
    assert rel(ge, demit) <= TOL, rel(ge, demit)


def test_autograd_function(torch_st):
    torch, st = torch_st
    wl = synth.gradient_problem(n_rays=1000)
    wl.n_bins = 32
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    k = torch.tensor(wl.k_band, device="cuda", requires_grad=True)
    m = torch.tensor(wl.mics, device="cuda", requires_grad=True)
    e = torch.tensor(wl.emitter, device="cuda", requires_grad=True)
    S = st.SpectraFn.apply(ctx, sc, p, k, m, e)
    loss = (S.abs() ** 2).sum()
    loss.backward()
    gk, gm, ge = ctx.backward(sc, 2.0 * S.detach(), k.shape[0], k.shape[1])
    # autograd forms dL/dS of |S|^2 through abs(), so it differs from 2 S by rounding only
    for a, b in ((k.grad, gk), (m.grad, gm), (e.grad, ge)):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-4 * float(b.abs().max()))


@pytest.mark.parametrize("mode", [0, 1])
def test_lobe_width_gradient_matches_oracle(torch_st, mode):
    """st_backward_beta against the oracle's float64 analytic gradient (itself pinned to central
    differences): both reflection modes, the clutter scene's four materials over 16 bands."""
    import oracle
    torch, st = torch_st
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=6, n_bins=40,
                       diffraction=False)
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance, reflection_mode=mode)
    S = ctx.simulate(sc, p)
    rng = np.random.default_rng(8)
    target = torch.as_tensor(rng.normal(size=S.shape) + 1j * rng.normal(size=S.shape), dtype=torch.complex64,
                             device=S.device) * S.abs().mean()
    G = 2.0 * (S - target)
    gb = ctx.backward_beta(sc, G, wl.k_band.shape[0], wl.k_band.shape[1]).cpu().numpy()
    o = oracle.simulate(wl, reflection_mode=mode)
    _, _, _, db = oracle.spectra_grad(o["params"], o["rec"], wl.dirs, wl.tri_mat,
                                      G.cpu().numpy().astype(np.complex128), direct_vis=o["direct_vis"],
                                      with_beta=True)
    assert np.abs(db).max() > 0
    assert rel(gb, db) <= TOL, rel(gb, db)


def test_autograd_lobe_widths(torch_st):
    torch, st = torch_st
    wl = synth.gradient_problem(n_rays=1000)
    wl.n_bins = 32
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    k = torch.tensor(wl.k_band, device="cuda")
    m = torch.tensor(wl.mics, device="cuda")
    e = torch.tensor(wl.emitter, device="cuda")
    b = torch.tensor(wl.beta_band, device="cuda", requires_grad=True)
    S = st.SpectraFn.apply(ctx, sc, p, k, m, e, b)
    (S.abs() ** 2).sum().backward()
    gb = ctx.backward_beta(sc, 2.0 * S.detach(), b.shape[0], b.shape[1])
    assert float(gb.abs().max()) > 0
    assert torch.allclose(b.grad, gb, rtol=1e-4, atol=1e-4 * float(gb.abs().max()))


def test_gradient_workload_full_size(torch_st):
    """The differentiation workload at its stated size: the four-material room, 10k rays x 3 bounces, the
    32-microphone disc array, 128 bins; gradients of the L2 loss against target spectra with respect to the
    4 x 16 reflection values and the 32 microphone positions (and the emitter) within 1e-3 of the oracle's
    float64 analytic gradient."""
    torch, st = torch_st
    wl = synth.gradient_problem(n_rays=10_000)
    assert wl.n_bins == 128 and len(wl.mics) == 32 and wl.k_band.shape == (4, 16)
    gk, gm, ge, dk, dmic, demit = grads_vs_oracle(torch, st, wl)
    assert rel(gk, dk) <= TOL, rel(gk, dk)
    assert rel(gm, dmic) <= TOL, rel(gm, dmic)
    assert rel(ge, demit) <= TOL, rel(ge, demit)


def test_backward_repeatable_after_chain_order(torch_st):
    """The first st_backward after a simulate puts the specular path list in reflection-chain order (paths with
    equal material counts side by side, gathered again); later backward calls find it in that order.  A second
    call gives bit-identical gradients, and the lobe-width gradient computed on the reordered list matches the
    one computed on the simulate's own order within float32 rounding."""
    torch, st = torch_st
    wl = synth.clutter(seed=202, target_tris=20_000, n_rays=20_000, bounces=4, n_mics=6, n_bins=40,
                       diffraction=False)
    n_mat, n_bands = wl.k_band.shape
    ctx = st.Context(0)
    sc = st.from_workload(ctx, wl)
    p = st.sim_params(max_bounces=wl.bounces, max_distance=wl.max_distance)
    S = ctx.simulate(sc, p)
    rng = np.random.default_rng(9)
    G = torch.as_tensor(rng.normal(size=S.shape) + 1j * rng.normal(size=S.shape), dtype=torch.complex64,
                        device=S.device)
    gb0 = ctx.backward_beta(sc, G, n_mat, n_bands).cpu().numpy()  # the simulate's order
    g1 = [g.cpu().numpy() for g in ctx.backward(sc, G, n_mat, n_bands)]
    g2 = [g.cpu().numpy() for g in ctx.backward(sc, G, n_mat, n_bands)]
    for a, b in zip(g1, g2):
        assert np.array_equal(a, b)
    gb1 = ctx.backward_beta(sc, G, n_mat, n_bands).cpu().numpy()  # the chain order
    assert np.abs(gb0).max() > 0
    assert rel(gb1, gb0) <= 1e-5, rel(gb1, gb0)
    # a new simulate starts from its own order again: the same gradients as the first call
    ctx.simulate(sc, p, out=S)
    g3 = [g.cpu().numpy() for g in ctx.backward(sc, G, n_mat, n_bands)]
    for a, b in zip(g1, g3):
        assert np.array_equal(a, b)
