"""The learned initial guess (kgs_net_*, kgs_surrogate_*) against the FP64
numpy reference of the same network (oracle/nn_ref.py) on the same
parameters and inputs.

The CUDA path stores weights and activations in bfloat16 and accumulates in
FP32; the reference sees the same bf16-rounded weights and stored activations
and computes in FP64.  The two differ by the FP32 accumulation order (about
1e-6 relative) and, where an FP32 and an FP64 sum fall on either side of a
bf16 rounding boundary, by one bf16 step (2^-8 relative) of that activation.
Outputs are compared to 2e-3 of their largest magnitude, the loss to 1e-4
relative.  The backward pass also stores the upstream gradients in bf16,
which the reference does not, so gradients are compared to 5e-2 in relative
L2 norm per tensor.
"""
import numpy as np
import pytest

from oracle import nn_ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def random_params(channels, seed):
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        W = rng.normal(0.0, np.sqrt(2.0 / (27 * cin)), size=(27, cout, cin))
        b = rng.normal(0.0, 0.1, size=cout)
        params.append((W, b))
    return params


def flat(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def unflat(vec, channels):
    out, k = [], 0
    for cin, cout in zip(channels[:-1], channels[1:]):
        W = vec[k:k + 27 * cout * cin].reshape(27, cout, cin)
        k += 27 * cout * cin
        out.append((W.astype(np.float64), vec[k:k + cout].astype(np.float64)))
        k += cout
    return out


def f32params(params):
    # the parameters as the GPU holds them in FP32 (before its bf16 rounding)
    return [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)) for W, b in params]


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("channels,shape", [
    ((11, 16, 112, 32, 8), (2, 5, 6, 7)),    # widest layer, ragged 4^3 tiles, two samples
    ((11, 48, 8), (1, 13, 9, 4)),            # odd extents, flat volume
])
def test_forward_matches_reference(kgs, channels, shape):
    params = random_params(channels, seed=1)
    net = kgs.kgs_net_create(channels, seed=0)
    kgs.kgs_net_set_params(net, flat(params))
    assert np.array_equal(kgs.kgs_net_get(net, 0), flat(params))
    rng = np.random.default_rng(2)
    x = rng.normal(size=shape + (channels[0],))
    xd = dev(x)
    yd = torch.empty(shape + (channels[-1],), device="cuda")
    kgs.kgs_net_forward(net, xd.data_ptr(), shape, yd.data_ptr())
    y = yd.cpu().numpy()
    p32 = f32params(params)
    for b in range(shape[0]):
        ref = nn_ref.forward(x[b].astype(np.float32), p32, bf16=True)[-1]
        scale = np.abs(ref).max()
        assert np.abs(y[b] - ref).max() <= 2e-3 * scale, (b, np.abs(y[b] - ref).max(), scale)


# Relative L2 errors of the weight and bias gradients per layer.  Both sides
# use the bf16-rounded weights and stored activations; the CUDA path also
# stores the propagated gradients in bf16, the reference keeps them in FP64;
# measured: at most 2.6e-3 on the first two cases, 1.6e-2 on the first layer
# of the full six-layer network (the gradient roundings accumulate over the
# depth of the backward pass).
@pytest.mark.parametrize("channels,shape,masked,tol", [
    ((11, 16, 112, 32, 8), (2, 5, 6, 7), False, 1e-2),
    ((11, 16, 8), (1, 20, 20, 20), True, 1e-2),     # 125 voxel tiles: several weight-gradient chunks
    ((11, 48, 112, 112, 112, 48, 8), (2, 16, 16, 16), False, 5e-2),  # the network the solver uses
])
def test_gradients_match_reference(kgs, channels, shape, masked, tol):
    params = random_params(channels, seed=3)
    net = kgs.kgs_net_create(channels, seed=0)
    kgs.kgs_net_set_params(net, flat(params))
    rng = np.random.default_rng(4)
    x = rng.normal(size=shape + (channels[0],))
    t = rng.normal(size=shape + (channels[-1],))
    mask = (rng.random(shape) < 0.7).astype(np.uint8) if masked else np.ones(shape, np.uint8)
    md = dev(mask, torch.uint8) if masked else None
    xd, td = dev(x), dev(t)   # kept alive until the step has run
    loss = kgs.kgs_net_train_step(net, xd.data_ptr(), td.data_ptr(), md.data_ptr() if masked else None,
                                  shape, lr=0.0)
    g = unflat(kgs.kgs_net_get(net, 1), channels)
    # parameters unchanged by an lr = 0 step
    assert np.array_equal(kgs.kgs_net_get(net, 0), flat(params))
    p32 = f32params(params)
    # reference over the whole batch: sum the per-sample gradients of the
    # batch-mean loss
    cnt = mask.sum() * channels[-1]
    ref_loss = 0.0
    ref_g = [(np.zeros_like(W), np.zeros_like(b)) for W, b in p32]
    for b in range(shape[0]):
        acts = nn_ref.forward(x[b].astype(np.float32), p32, bf16=True)
        d = (acts[-1] - t[b].astype(np.float32)) * mask[b][..., None]
        ref_loss += float((d * d).sum()) / cnt
        gb = nn_ref.backward(acts, p32, 2.0 * d / cnt, bf16=True)
        ref_g = [(rW + gW, rb + gbb) for (rW, rb), (gW, gbb) in zip(ref_g, gb)]
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss, (loss, ref_loss)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(g, ref_g)):
        eW = np.linalg.norm(gW - rW) / np.linalg.norm(rW)
        eb = np.linalg.norm(gb - rb) / np.linalg.norm(rb)
        assert eW <= tol and eb <= tol, (l, eW, eb)


def test_training_reduces_loss(kgs):
    channels = (11, 32, 32, 8)
    shape = (2, 8, 8, 8)
    net = kgs.kgs_net_create(channels, seed=5)
    rng = np.random.default_rng(6)
    x = dev(rng.normal(size=shape + (11,)))
    # a target the network can represent: a smooth function of the inputs
    xs = x.cpu().numpy()
    t = np.stack([np.tanh(xs[..., c] + 0.5 * xs[..., c + 1]) for c in range(8)], axis=-1)
    td = dev(t)
    losses = [kgs.kgs_net_train_step(net, x.data_ptr(), td.data_ptr(), None, shape, lr=3e-3) for _ in range(60)]
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0], losses[::10]


def test_features_target_apply(kgs):
    nx, ny, nz, nxc, nyc, nzc = 10, 7, 6, 5, 4, 3
    rng = np.random.default_rng(8)
    coarse = rng.normal(size=(8, nzc, nyc, nxc)) * 0.05
    coarse[0] += 1.0
    coarse[4] += 1.0
    solid = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8)
    x = torch.empty((nz, ny, nx, 11), device="cuda")
    up = torch.empty((8, nz, ny, nx), dtype=torch.float64, device="cuda")
    cd = dev(coarse, torch.float64)
    sd = dev(solid, torch.uint8)
    kgs.kgs_surrogate_features((nx, ny, nz), (nxc, nyc, nzc), cd.data_ptr(), sd.data_ptr(), 0.2, 0.16,
                               x.data_ptr(), up.data_ptr())
    torch.cuda.synchronize()

    # separable linear interpolation between cell centres, clamped at the ends
    def axis(n, nc):
        return (np.arange(n) + 0.5) / n * nc - 0.5

    ref = coarse
    for ax, (n, nc) in zip((3, 2, 1), ((nx, nxc), (ny, nyc), (nz, nzc))):
        ref = np.apply_along_axis(lambda v: np.interp(axis(n, nc), np.arange(nc), v), ax, ref)
    upn = up.cpu().numpy()
    assert np.abs(upn - ref).max() < 1e-14
    xn = x.cpu().numpy().astype(np.float64)
    scale = np.array([10, 10, 10, 10, 50, 100, 100, 100], np.float64)
    rest = np.array([1, 0, 0, 0, 1, 0, 0, 0], np.float64)
    assert np.allclose(xn[..., 0], np.log(0.2), rtol=1e-6)
    assert np.allclose(xn[..., 1], 1.6, rtol=1e-6)
    assert np.array_equal(xn[..., 2], solid.astype(np.float64))
    norm = (np.moveaxis(ref, 0, -1) - rest) * scale
    assert np.allclose(xn[..., 3:], norm, rtol=1e-6, atol=1e-6)

    fine = ref + rng.normal(size=ref.shape) * 1e-3
    tg = torch.empty((nz * ny * nx, 8), device="cuda")
    fd = dev(fine, torch.float64)
    kgs.kgs_surrogate_target(nx * ny * nz, fd.data_ptr(), up.data_ptr(), tg.data_ptr())
    tn = tg.cpu().numpy().astype(np.float64)
    assert np.allclose(tn, (fine - ref).reshape(8, -1).T * scale, rtol=1e-6, atol=1e-7)

    # applying the exact correction recovers the fine field; a guess with a
    # non-positive density or temperature is counted as bad
    m = torch.empty((8, nz, ny, nx), dtype=torch.float64, device="cuda")
    assert kgs.kgs_surrogate_apply(nx * ny * nz, up.data_ptr(), tg.data_ptr(), m.data_ptr()) == 0
    assert np.abs(m.cpu().numpy() - fine).max() < 1e-7
    bad = tg.clone()
    bad[3, 0] = -1e3       # rho of cell 3 below zero
    bad[5, 4] = float("nan")
    assert kgs.kgs_surrogate_apply(nx * ny * nz, up.data_ptr(), bad.data_ptr(), m.data_ptr()) == 2
