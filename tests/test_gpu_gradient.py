"""The hand-written backward kernel (through the C ABI and the
torch.autograd.Function) against the binary64 oracle gradient and against
binary64 central finite differences; the 64-cloud gradient-descent
configuration (N=2048, d=3, loss = sum of squared deaths, 100 steps)."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ph0():
    from paper_2203_02527_gb300 import ph0
    return ph0


def test_backward_matches_fp64_reference_gradient():
    ph0 = _ph0()
    x = inputs.uniform(2048, 3, seed=81)
    pts = torch.from_numpy(x).cuda().requires_grad_(True)
    deaths = ph0.death_values(pts)
    loss = (deaths ** 2).sum()
    loss.backward()
    bars = oracle.barcodes(x)[0]
    ref = oracle.death_gradient(x.astype(np.float64), bars["u"], bars["v"], 2.0 * bars["death"])
    got = pts.grad.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6 * scale)
    # the forward values are the oracle's deaths, bit for bit
    np.testing.assert_array_equal(deaths.detach().cpu().numpy().view(np.uint64),
                                  bars["death"].view(np.uint64))


def test_backward_matches_central_finite_differences():
    ph0 = _ph0()
    x = inputs.uniform(120, 3, seed=82)
    pts = torch.from_numpy(x).cuda().requires_grad_(True)
    (ph0.death_values(pts) ** 2).sum().backward()
    g = pts.grad.cpu().numpy().astype(np.float64)
    x64 = x.astype(np.float64)
    _, u0, v0, _ = oracle.barcodes_f64(x64)
    key0 = np.sort(u0.astype(np.int64) * 65536 + v0)
    h = 1e-4
    rng = np.random.default_rng(5)
    checked = skipped = 0
    for idx in rng.choice(x.size, 80, replace=False):
        i, k = divmod(int(idx), x.shape[1])
        xp, xm = x64.copy(), x64.copy()
        xp[i, k] += h
        xm[i, k] -= h
        sp, sm = oracle.barcodes_f64(xp), oracle.barcodes_f64(xm)
        if not all(np.array_equal(np.sort(s[1].astype(np.int64) * 65536 + s[2]), key0) for s in (sp, sm)):
            skipped += 1  # the pairing changes within the step (a tie): not differentiable there
            continue
        fd = (sp[3].sum() - sm[3].sum()) / (2 * h)
        assert abs(g[i, k] - fd) <= 1e-4 * max(abs(fd), 1e-3), (i, k, g[i, k], fd)
        checked += 1
    assert checked >= 60, (checked, skipped)


def test_backward_general_upstream_gradient_and_zero_length_bars():
    ph0 = _ph0()
    x = inputs.with_duplicates(300, 3, 200, seed=83)  # duplicates: bars of length 0
    pts = torch.from_numpy(x).cuda()
    bars = ph0.barcodes(pts)
    w = torch.linspace(-1.0, 2.0, 299, dtype=torch.float64, device="cuda")
    g = ph0.backward(pts, bars, w).cpu().numpy().astype(np.float64)
    ob = oracle.barcodes(x)[0]
    ref = oracle.death_gradient(x.astype(np.float64), ob["u"], ob["v"], w.cpu().numpy())
    np.testing.assert_allclose(g, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_gradient_descent_64_clouds():
    """64 clouds, N=2048, d=3, U[0,1)^3; 100 steps of gradient descent on the
    coordinates with loss = sum of squared finite deaths (learning rate 1e-2)."""
    ph0 = _ph0()
    clouds = [torch.from_numpy(inputs.uniform(2048, 3, seed=1000 + c)).cuda().requires_grad_(True)
              for c in range(64)]
    ws = ph0.Workspace(2048, 3)
    opt = torch.optim.SGD(clouds, lr=1e-2)
    losses = []
    for step in range(100):
        opt.zero_grad()
        total = sum((ph0.death_values(p, ws) ** 2).sum() for p in clouds)
        total.backward()
        opt.step()
        losses.append(float(total.detach()))
    assert losses[-1] < losses[0]
    assert all(np.isfinite(losses))
    # after the descent the gradient of one cloud still matches the reference
    p = clouds[7].detach().clone().requires_grad_(True)
    (ph0.death_values(p, ws) ** 2).sum().backward()
    x = p.detach().cpu().numpy()
    ob = oracle.barcodes(x)[0]
    ref = oracle.death_gradient(x.astype(np.float64), ob["u"], ob["v"], 2.0 * ob["death"])
    np.testing.assert_allclose(p.grad.cpu().numpy(), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_batched_death_values_equal_one_at_a_time():
    """The batched form (clouds on several streams) gives the same deaths and
    gradients as one call per cloud."""
    ph0 = _ph0()
    xs = [inputs.uniform(700 + 37 * c, 3, seed=2000 + c) for c in range(12)]
    batch = ph0.Batch([x.shape for x in xs], streams=4)
    pts = [torch.from_numpy(x).cuda().requires_grad_(True) for x in xs]
    deaths = batch.death_values(pts)
    sum((dv ** 2).sum() for dv in deaths).backward()
    for x, p, dv in zip(xs, pts, deaths):
        q = torch.from_numpy(x).cuda().requires_grad_(True)
        one = ph0.death_values(q)
        assert torch.equal(one, dv)
        (one ** 2).sum().backward()
        np.testing.assert_allclose(p.grad.cpu().numpy(), q.grad.cpu().numpy(), rtol=1e-6, atol=1e-9)


def test_captured_batched_step_replays_the_eager_steps():
    """The batched descent step captured once into a CUDA graph and replayed
    follows the eager trajectory: the same deaths at every step (the pairing
    and distances are exact), the points within the last bit of the binary64
    gradient sums (accumulated by atomics in any order), and the statuses of
    every cloud read in one copy after each replay."""
    ph0 = _ph0()
    xs = [inputs.uniform(600 + 50 * c, 3, seed=3000 + c) for c in range(10)]

    def trajectory(graphed):
        pts = [torch.from_numpy(x).cuda().requires_grad_(True) for x in xs]
        opt = torch.optim.SGD(pts, lr=1e-2)
        batch = ph0.Batch([x.shape for x in xs], streams=4)
        losses = []

        def step():
            deaths = batch.death_values(pts)
            total = sum((dv ** 2).sum() for dv in deaths)
            total.backward()
            opt.step()
            return total

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                opt.zero_grad(set_to_none=True)
                losses.append(float(step().detach()))
        torch.cuda.current_stream().wait_stream(side)
        if graphed:
            graph = torch.cuda.CUDAGraph()
            opt.zero_grad(set_to_none=True)
            with torch.cuda.graph(graph):
                static_total = step()
            for _ in range(5):
                graph.replay()
                losses.append(float(static_total.detach()))
                batch.check()
        else:
            for _ in range(5):
                opt.zero_grad(set_to_none=True)
                losses.append(float(step().detach()))
        return losses, [p.detach().cpu().numpy() for p in pts]

    l_eager, p_eager = trajectory(False)
    l_graph, p_graph = trajectory(True)
    np.testing.assert_allclose(l_graph, l_eager, rtol=1e-9)
    for a, b in zip(p_graph, p_eager):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-6)
    assert l_graph[-1] < l_graph[0]
