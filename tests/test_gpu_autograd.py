"""Differentiable solve (quantise -> solve -> one-hot backward, structured hinge) against
the oracle and brute force. Every compared value is an integer in quantised units or a
gradient entry in {-1, 0, 1}: tolerance 0."""
import numpy as np
import pytest

import oracle
import pins
from paper_2601_17026_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2601_17026_gb300 import autograd as pag  # noqa: E402
from paper_2601_17026_gb300 import pog  # noqa: E402

SCALE = 1024.0


def quantise(c):
    return np.rint(np.asarray(c, dtype=np.float64) * SCALE).astype(np.int32)


def onehot(h, Z):
    h = np.asarray(h)
    return (np.arange(Z)[None, None, None, :] == h[..., None]).astype(np.float32)


def test_backward_kernel_formula():
    rng = np.random.default_rng(1)
    B, X, Y, Z = 3, 5, 7, 9
    h, ht, hh = (rng.integers(0, Z, size=(B, X, Y)).astype(np.int32) for _ in range(3))
    ge = rng.standard_normal(B).astype(np.float32)
    gh = rng.standard_normal(B).astype(np.float32)
    grad = torch.full((B, X, Y, Z), 7.0, device="cuda")
    t = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    pog.pog_backward(grad, t(h), t(ge), t(ht), t(hh), t(gh))
    want = ge[:, None, None, None] * onehot(h, Z) + gh[:, None, None, None] * (onehot(ht, Z) - onehot(hh, Z))
    np.testing.assert_array_equal(grad.cpu().numpy(), want)
    grad2 = torch.full((B, X, Y, Z), 7.0, device="cuda")
    pog.pog_backward(grad2, t(h), t(ge))
    np.testing.assert_array_equal(grad2.cpu().numpy(), ge[:, None, None, None] * onehot(h, Z))


def test_energy_and_gradient_match_oracle():
    specs = [synth.scaled_spec(12, 10, 16, 100 + i, stream=3000 + i) for i in range(3)]
    fc = np.stack([synth.float_horizon_cost(s) for s in specs])
    x = torch.from_numpy(fc).cuda().requires_grad_(True)
    e = pag.pog_energy(x, delta=2, alpha=10.0)
    e.sum().backward()
    grad = x.grad.cpu().numpy()
    for b in range(len(specs)):
        cq = quantise(fc[b])
        ref = oracle.solve(cq, 2, 10240)
        eq, ok = oracle.energy(cq, ref.heights, 2, 10240)
        assert ok
        assert e[b].item() * SCALE == eq
        np.testing.assert_array_equal(grad[b], onehot(ref.heights[None], 16)[0])


def _unique_tiny(rng, shape, delta, alpha_q, margin=2):
    """Tiny float volume whose quantised problem has a unique optimum by >= margin."""
    for _ in range(200):
        c = (rng.integers(-60, 60, size=shape) / SCALE * 7).astype(np.float32)
        cq = quantise(c)
        emin, hmin, opt = pins.brute_force(cq, delta, alpha_q)
        if len(opt) != 1:
            continue
        # second best energy over all feasible surfaces
        X, Y, Z = shape
        import itertools

        best2 = None
        for hs in itertools.product(range(Z), repeat=X * Y):
            h = np.array(hs).reshape(X, Y)
            if not pins.feasible(h, delta) or np.array_equal(h, hmin):
                continue
            ev = pins.energy(cq, h, alpha_q)
            best2 = ev if best2 is None else min(best2, ev)
        if best2 is None or best2 - emin >= margin:
            return c, cq, emin, hmin
    raise RuntimeError("no uniquely optimal volume found")


def test_finite_differences_exact():
    """(E*(c + e) - E*(c - e)) / 2 equals the one-hot gradient at e, with e one quantum."""
    rng = np.random.default_rng(5)
    delta, alpha = 1, 2.0
    aq = int(alpha * SCALE)
    c, cq, emin, hmin = _unique_tiny(rng, (2, 3, 4), delta, aq)
    x = torch.from_numpy(c[None]).cuda().requires_grad_(True)
    e = pag.pog_energy(x, delta=delta, alpha=alpha)
    assert e.item() * SCALE == emin
    e.backward()
    g = x.grad.cpu().numpy()[0]
    for idx in np.ndindex(c.shape):
        up = c.copy()
        dn = c.copy()
        up[idx] += np.float32(1.0 / SCALE)
        dn[idx] -= np.float32(1.0 / SCALE)
        assert quantise(up)[idx] == cq[idx] + 1 and quantise(dn)[idx] == cq[idx] - 1
        ep = pag.pog_energy(torch.from_numpy(up[None]).cuda(), delta=delta, alpha=alpha).item() * SCALE
        em = pag.pog_energy(torch.from_numpy(dn[None]).cuda(), delta=delta, alpha=alpha).item() * SCALE
        assert (ep - em) / 2 == g[idx]


def _brute_hinge(cq, ht, delta, aq, mq):
    """min over feasible h of E(h) - mq * Hamming(h, ht), its lowest minimiser, and E(ht)."""
    X, Y, Z = cq.shape
    import itertools

    best, arg = None, []
    for hs in itertools.product(range(Z), repeat=X * Y):
        h = np.array(hs).reshape(X, Y)
        if not pins.feasible(h, delta):
            continue
        v = pins.energy(cq, h, aq) - mq * int((h != ht).sum())
        if best is None or v < best:
            best, arg = v, [h]
        elif v == best:
            arg.append(h)
    return best, np.min(np.stack(arg), axis=0), pins.energy(cq, ht, aq)


def test_hinge_loss_and_gradient_brute_force():
    rng = np.random.default_rng(9)
    delta, alpha, margin = 1, 1.0, 1.0
    aq, mq = int(alpha * SCALE), int(margin * SCALE)
    for _ in range(4):
        c = (rng.integers(-40, 40, size=(2, 3, 4)) / SCALE * 37).astype(np.float32)
        cq = quantise(c)
        ht = pins.brute_force(quantise(rng.standard_normal((2, 3, 4)).astype(np.float32)), delta, aq)[1]
        best, hhat, et = _brute_hinge(cq, ht, delta, aq, mq)
        x = torch.from_numpy(c[None]).cuda().requires_grad_(True)
        e, loss, h, hh = pag.solve_with_hinge(x, torch.from_numpy(ht[None].astype(np.int32)).cuda(), delta, alpha,
                                              margin)
        assert loss.item() * SCALE == et - best
        np.testing.assert_array_equal(hh.cpu().numpy()[0], hhat)
        loss.sum().backward()
        np.testing.assert_array_equal(x.grad.cpu().numpy()[0], onehot(ht[None], 4)[0] - onehot(hhat[None], 4)[0])


def test_hinge_against_oracle_on_augmented_costs():
    specs = [synth.scaled_spec(24, 20, 32, 200 + i, stream=4000 + i) for i in range(2)]
    fc = np.stack([synth.float_horizon_cost(s) for s in specs])
    # targets: the oracle's surfaces of the same recipe with the next seed
    hts = []
    for s in specs:
        other = synth.float_horizon_cost(synth.scaled_spec(s.X, s.Y, s.Z, s.seed + 1, stream=s.stream))
        hts.append(oracle.solve(quantise(other), 2, 10240).heights)
    ht = np.stack(hts).astype(np.int32)
    x = torch.from_numpy(fc).cuda().requires_grad_(True)
    e, loss, h, hh = pag.solve_with_hinge(x, torch.from_numpy(ht).cuda(), 2, 10.0, 1.0)
    (e.sum() + 3.0 * loss.sum()).backward()
    grad = x.grad.cpu().numpy()
    for b in range(2):
        cq = quantise(fc[b])
        aug = cq.copy()
        np.put_along_axis(aug, ht[b][:, :, None], np.take_along_axis(cq, ht[b][:, :, None], 2) + 1024, axis=2)
        ref_aug = oracle.solve(aug, 2, 10240)
        np.testing.assert_array_equal(hh.cpu().numpy()[b], ref_aug.heights)
        ref = oracle.solve(cq, 2, 10240)
        np.testing.assert_array_equal(h.cpu().numpy()[b], ref.heights)
        et, _ = oracle.energy(cq, ht[b], 2, 10240)
        eaug, _ = oracle.energy(aug, ref_aug.heights, 2, 10240)
        assert loss[b].item() * SCALE == et - (eaug - 1024 * 24 * 20)
        Z = 32
        want = onehot(ref.heights[None], Z)[0] + 3.0 * (onehot(ht[b][None], Z)[0] - onehot(ref_aug.heights[None], Z)[0])
        np.testing.assert_array_equal(grad[b], want)


def test_surface_energy_kernel():
    spec = synth.scaled_spec(16, 12, 20, 7, stream=5000)
    fc = synth.float_horizon_cost(spec)[None]
    rng = np.random.default_rng(3)
    h = rng.integers(0, 20, size=(1, 16, 12)).astype(np.int32)
    out = pog.pog_surface_energy(torch.from_numpy(fc).cuda(), SCALE, torch.from_numpy(h).cuda(), 300).cpu().numpy()
    assert out[0] == pins.energy(quantise(fc[0]), h[0], 300)
    h[0, 0, 0] = 20  # outside [0, Z)
    out = pog.pog_surface_energy(torch.from_numpy(fc).cuda(), SCALE, torch.from_numpy(h).cuda(), 300).cpu().numpy()
    assert out[0] == np.iinfo(np.int64).min


@pytest.mark.parametrize("target", ["random", "bottom", "top", "mixed"])
def test_warm_hinge_matches_cold_and_oracle(target):
    """The loss-augmented solve started from the energy solve's final state gives the
    oracle's flow, energy and surface of the augmented problem, including targets on the
    bottom layer (its constants change) and on the top layer (no node above it)."""
    rng = np.random.default_rng({"random": 1, "bottom": 2, "top": 3, "mixed": 4}[target])
    specs = [synth.scaled_spec(20, 17, 24, 300 + i, stream=6000 + i) for i in range(3)]
    fc = np.stack([synth.float_horizon_cost(s) for s in specs])
    B, X, Y, Z = fc.shape
    if target == "random":
        ht = rng.integers(0, Z, size=(B, X, Y))
    elif target == "bottom":
        ht = np.zeros((B, X, Y))
    elif target == "top":
        ht = np.full((B, X, Y), Z - 1)
    else:
        ht = rng.choice([0, 1, Z - 2, Z - 1, Z // 2], size=(B, X, Y))
    ht = ht.astype(np.int32)
    delta, aq, mq = 2, 10240, 3000
    xc = torch.from_numpy(fc).cuda()
    htd = torch.from_numpy(ht).cuda()
    outs = [pog.pog_solve_batch_f32_hinge(xc, SCALE, htd, mq, delta, aq, pog.make_options(flags=f))
            for f in (0, pog.POG_FLAG_COLD_HINGE)]
    for b in range(B):
        cq = quantise(fc[b])
        aug = cq.copy()
        np.put_along_axis(aug, ht[b][:, :, None], np.take_along_axis(cq, ht[b][:, :, None], 2) + mq, axis=2)
        ref = oracle.solve(cq, delta, aq)
        ref_aug = oracle.solve(aug, delta, aq)
        e_aug, _ = oracle.energy(aug, ref_aug.heights, delta, aq)
        e_t, _ = oracle.energy(cq, ht[b], delta, aq)
        for out in outs:
            assert out["flows"][b] == ref.flow
            assert out["aug_flows"][b] == ref_aug.flow
            assert out["aug_energies"][b] == e_aug
            assert out["hinge"][b] == e_t - (e_aug - mq * X * Y)
            np.testing.assert_array_equal(out["heights"][b].cpu().numpy(), ref.heights)
            np.testing.assert_array_equal(out["h_hat"][b].cpu().numpy(), ref_aug.heights)


def test_hinge_rejects_targets_outside_the_volume():
    fc = torch.zeros((1, 4, 5, 6), device="cuda")
    ht = torch.zeros((1, 4, 5), dtype=torch.int32, device="cuda")
    ht[0, 1, 2] = 6
    with pytest.raises(pog.PogError) as ei:
        pog.pog_solve_batch_f32_hinge(fc, SCALE, ht, 1024, 1, 0)
    assert ei.value.status == pog.POG_E_INVALID


def test_int32_headroom_on_the_differentiable_scale():
    """Excess and arc flows are int32 words (checked adds, POG_E_OVERFLOW on a wrap). On a
    128^3 volume of the differentiable workload (quantised costs up to about 1.03M,
    alpha 10240) the final state stays far inside int32: every excess, sink residual and
    finite arc flow below 2^25, i.e. at least 64x of headroom (measured peaks on the first
    four volumes: 3.4-6.3 M)."""
    fc = synth.diff_volumes_f32(count=1)
    t = torch.from_numpy(fc[0]).cuda()
    with pog.pog_build_f32(t, SCALE, synth.DIFF_DELTA, int(synth.DIFF_ALPHA * SCALE)) as g:
        pog.pog_maxflow(g)
        st = pog.pog_export_state(g)
    peak = max(int(np.abs(st[k]).max()) for k in ("excess", "sink", "fdown", "fhard", "gsoft"))
    assert 0 < peak < (1 << 25), peak
