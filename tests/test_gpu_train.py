"""GPU tests of the fused training pass exw_warp_l2_grad (the warp of stage (b) inside an L2 loss, P_1..P_3, with
its adjoint): bit-identical gradients to the staged entry points (splat, warp, L2 loss, adjoint per fraction),
gradients within 1e-5 + 1e-4 relative of the FP64 oracle's, and central finite differences (eps 1e-3, FP64 oracle
loss) of the loss on a 64 x 64 crop of the differentiation workload, skipping perturbations that change an integer
decision (a target, a winner or the side of a tap)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2307_12607_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the gpu-marked tests")
    from paper_2307_12607_gb300 import build, binding
    build.build()
    return binding


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def grad_close(got, want, what=""):
    got = got.astype(np.float64)
    err = np.abs(got - want)
    bound = 1e-5 + 1e-4 * np.abs(want)
    assert np.all(err <= bound), f"{what}: max excess {np.max(err - bound)}"


def frames_and_targets(W, H, nframes, seed, dtype=np.float32):
    s = scenes.make_scene(W, H, seed, 10, vmax=8.0, pan_max=3.0, sliver_fraction=0.2)
    fr = [scenes.render(s, float(f)) for f in range(nframes)]
    tg = [[scenes.ground_truth(s, float(f), k) for k in (1, 2, 3)] for f in range(nframes)]
    col = np.stack([f[0] for f in fr]).astype(dtype)
    dep = np.stack([f[1] for f in fr])
    mv = np.stack([f[2] for f in fr])
    targets = np.stack([np.stack(t) for t in tg]).astype(dtype)
    return col, dep, mv, targets


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
@pytest.mark.parametrize("nfrac", [3, 1])
def test_fused_pass_equals_staged_entry_points(b, dtype, nfrac):
    col, dep, mv, tg = frames_and_targets(257, 131, 3, 51, dtype)
    c, d, m, t = dev(col), dev(dep), dev(mv), dev(tg[:, :nfrac])
    gc0 = torch.randn((3, 3, 131, 257), device="cuda")     # the gradients accumulate into what is there
    gm0 = torch.randn((3, 2, 131, 257), device="cuda")
    loss, gc, gm = b.exw_warp_l2_grad(c, d, m, t, nfrac, grad_color=gc0.clone(), grad_mv=gm0.clone())
    for f in range(3):
        sgc, sgm = gc0[f].clone(), gm0[f].clone()
        lsum = torch.zeros(1, device="cuda")
        for k in range(1, nfrac + 1):
            keys = b.exw_splat_motion(d[f], m[f], k, 4)
            out, mask = b.exw_warp(c[f], d[f], m[f], keys, k, 4)
            _, g = b.exw_l2_loss_grad(out, t[f, k - 1], mask, loss=lsum)
            b.exw_warp_backward(g, c[f], d[f], m[f], None, k, 4, sgc, sgm)
        assert torch.equal(gc[f], sgc) and torch.equal(gm[f], sgm), f"frame {f}"
        assert loss[f].item() == pytest.approx(lsum.item(), rel=1e-5)
    # deterministic: a second call gives the same bits
    loss2, gc2, gm2 = b.exw_warp_l2_grad(c, d, m, t, nfrac, grad_color=gc0.clone(), grad_mv=gm0.clone())
    assert torch.equal(loss2, loss) and torch.equal(gc2, gc) and torch.equal(gm2, gm)


@pytest.mark.parametrize("case", [(257, 131, 52), (96, 64, 53), (33, 17, 54)])
def test_fused_pass_matches_oracle(b, case):
    W, H, seed = case
    col, dep, mv, tg = frames_and_targets(W, H, 2, seed)
    loss, gc, gm = b.exw_warp_l2_grad(dev(col), dev(dep), dev(mv), dev(tg), 3)
    for f in range(2):
        wl, wc, wm = 0.0, np.zeros((3, H, W)), np.zeros((2, H, W))
        for k in (1, 2, 3):
            keys = oracle.splat(dep[f], mv[f], k)
            out, mask = oracle.warp(col[f].astype(np.float64), dep[f], mv[f], keys, k)
            lk, g = oracle.l2_loss_grad(out, tg[f, k - 1], mask)
            wl += lk
            wc, wm = oracle.warp_backward(g, col[f].astype(np.float64), dep[f], mv[f], keys, k, grad_color=wc,
                                          grad_mv=wm)
        assert loss[f].item() == pytest.approx(wl, rel=1e-5, abs=1e-9)
        grad_close(gc[f].cpu().numpy(), wc, f"colour gradient, frame {f}")
        grad_close(gm[f].cpu().numpy(), wm, f"motion gradient, frame {f}")


def _rho_signs(mv, keys, k):
    """Side of each winner's taps (sign of rho per axis) -- exact in FP64 (an integer minus a float32 times k/4)."""
    H, W = keys.shape
    q = np.flatnonzero(keys.ravel() != oracle.EMPTY)
    p = (keys.ravel()[q] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    sig = np.zeros((2, H, W), np.int8)
    for a, (t, s) in enumerate(((q % W, p % W), (q // W, p // W))):
        rho = (t - s).astype(np.float64) - mv[a].ravel()[p].astype(np.float64) * k / 4
        sig[a].ravel()[q] = np.sign(rho).astype(np.int8)
    return sig


def _oracle_loss(color, depth, mv, targets):
    """The FP64 oracle's loss over the three fractions and its integer decisions (keys, tap sides)."""
    total, dec = 0.0, []
    for k in (1, 2, 3):
        keys = oracle.splat(depth, mv, k)
        out, mask = oracle.warp(color, depth, mv, keys, k)
        total += oracle.l2_loss_grad(out, targets[k - 1], mask)[0]
        dec.append((keys, _rho_signs(mv, keys, k)))
    return total, dec


def _same_decisions(d0, d1):
    return all(np.array_equal(a[0], b_[0]) and np.array_equal(a[1], b_[1]) for a, b_ in zip(d0, d1))


def test_central_differences_on_a_crop_of_the_differentiation_workload(b):
    # a 64 x 64 crop of the 1920 x 1080 differentiation scene at the place with the most distinct motions (object
    # edges, holes), targets = the scene rendered at t + k/4
    s = scenes.diff_scene()
    color, depth, mv = scenes.render(s, 0.0)
    gts = [scenes.ground_truth(s, 0.0, k) for k in (1, 2, 3)]
    best, at = -1, (0, 0)
    for y0 in range(0, 1080 - 64, 32):
        for x0 in range(0, 1920 - 64, 32):
            n = len(np.unique(mv[0, y0:y0 + 64, x0:x0 + 64]))
            if n > best:
                best, at = n, (y0, x0)
    y0, x0 = at
    crop = lambda a: np.ascontiguousarray(a[..., y0:y0 + 64, x0:x0 + 64])
    c, d, m = crop(color), crop(depth), crop(mv)
    tg = np.stack([crop(g) for g in gts])
    loss, gc, gm = b.exw_warp_l2_grad(dev(c[None]), dev(d[None]), dev(m[None]), dev(tg[None]), 3)
    gc, gm = gc[0].cpu().numpy().astype(np.float64), gm[0].cpu().numpy().astype(np.float64)
    C = c.astype(np.float64)
    l0, dec0 = _oracle_loss(C, d, m, tg)
    assert loss[0].item() == pytest.approx(l0, rel=1e-5)
    rng = np.random.default_rng(7)
    # motion: central differences with eps = 1e-3 in float32, skipping a perturbation that changes a decision
    checked = 0
    for idx in rng.choice(2 * 64 * 64, 240, replace=False):
        a, p = divmod(int(idx), 64 * 64)
        vals = []
        for sgn in (1, -1):
            mp = m.copy()
            mp[a].flat[p] = np.float32(m[a].flat[p] + sgn * 1e-3)
            lv, dec = _oracle_loss(C, d, mp, tg)
            if not _same_decisions(dec, dec0):
                vals = None
                break
            vals.append((lv, float(mp[a].flat[p])))
        if vals is None:
            continue
        (lp, xp), (lm, xm) = vals
        fd = (lp - lm) / (xp - xm)
        assert abs(fd - gm[a].flat[p]) <= 1e-5 + 1e-4 * abs(fd), (a, p, fd, gm[a].flat[p])
        checked += 1
    assert checked > 150
    # colour: the loss is quadratic in the colour, so central differences are exact up to rounding
    for idx in rng.choice(3 * 64 * 64, 120, replace=False):
        e = 1e-3
        Cp, Cm = C.copy(), C.copy()
        Cp.flat[idx] += e
        Cm.flat[idx] -= e
        fd = (_oracle_loss(Cp, d, m, tg)[0] - _oracle_loss(Cm, d, m, tg)[0]) / (2 * e)
        assert abs(fd - gc.flat[idx]) <= 1e-5 + 1e-4 * abs(fd), (idx, fd, gc.flat[idx])
