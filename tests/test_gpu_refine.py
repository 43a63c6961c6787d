"""GPU parity of the differentiable refinement form against the FP64 oracle:
FP32 forward/backward (through plan_refine and the autograd.Function) vs the
FP64 loss and analytic gradient, plus central finite differences of the GPU
loss.  Bar: loss within 1e-4 relative; gradient relative L2 error per
segment with median <= 1e-4 and max <= 1e-2 (reported)."""
import numpy as np
import pytest

from oracle import refine as OR
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import refine as RF  # noqa: E402


def dev(rb):
    f = lambda x: torch.as_tensor(np.asarray(x, dtype=np.float32)).cuda().contiguous()
    return (f(rb.P), f(rb.T), f(rb.A), f(rb.b), torch.as_tensor(rb.nrows, dtype=torch.int32).cuda())


def rel_l2(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


@pytest.mark.parametrize("S", [1, 1000, 65536])
def test_refine_forward_backward_vs_fp64(S):
    rb = synth.refine_segments(seed=5, S=S)
    P32 = rb.P.astype(np.float32).astype(np.float64)
    T32 = rb.T.astype(np.float32).astype(np.float64)
    A32 = rb.A.astype(np.float32).astype(np.float64)
    b32 = rb.b.astype(np.float32).astype(np.float64)
    ref_l, ref_dP, ref_dT = OR.loss_and_grad(P32, T32, A32, b32, rb.nrows, rb.bounds)
    refiner = RF.Refiner()
    P, T, A, b, nr = dev(rb)
    P.requires_grad_(True)
    T.requires_grad_(True)
    loss = RF.refine_loss(P, T, A, b, nr, refiner)
    up = torch.ones_like(loss)
    loss.backward(up)
    refiner.check()
    gl = loss.detach().cpu().numpy().astype(np.float64)
    rel_loss = np.abs(gl - ref_l) / np.maximum(np.abs(ref_l), 1.0)
    assert rel_loss.max() <= 1e-4, rel_loss.max()
    g = np.concatenate([P.grad.cpu().numpy().reshape(S, -1), T.grad.cpu().numpy()[:, None]], axis=1).astype(np.float64)
    r = np.concatenate([ref_dP.reshape(S, -1), ref_dT[:, None]], axis=1)
    e = rel_l2(g, r)
    print(f"S={S}: grad rel-L2 median {np.median(e):.2e} max {e.max():.2e}; loss rel max {rel_loss.max():.2e}")
    assert np.median(e) <= 1e-4 and e.max() <= 1e-2


def test_refine_upstream_gradient_scaling_and_zero_rows():
    rb = synth.refine_segments(seed=8, S=300)
    rb.nrows[:50] = 0
    refiner = RF.Refiner()
    P, T, A, b, nr = dev(rb)
    w = torch.linspace(-2.0, 3.0, 300, device="cuda")
    dP, dT = refiner.backward(P, T, A, b, nr, w)
    refiner.check()
    ref_l, ref_dP, ref_dT = OR.loss_and_grad(rb.P.astype(np.float32).astype(np.float64),
                                             rb.T.astype(np.float32).astype(np.float64),
                                             rb.A.astype(np.float32).astype(np.float64),
                                             rb.b.astype(np.float32).astype(np.float64), rb.nrows, rb.bounds)
    wn = w.cpu().numpy().astype(np.float64)
    e = rel_l2(dP.cpu().numpy().reshape(300, -1), ref_dP.reshape(300, -1) * wn[:, None])
    assert np.median(e) <= 1e-4
    np.testing.assert_allclose(dT.cpu().numpy(), ref_dT * wn, rtol=1e-3, atol=1e-3)


def test_refine_gpu_loss_finite_differences():
    """Central differences of the GPU loss itself (FP32, h chosen for FP32)."""
    rb = synth.refine_segments(seed=4, S=64)
    refiner = RF.Refiner()
    P, T, A, b, nr = dev(rb)
    dP, dT = refiner.backward(P, T, A, b, nr, torch.ones(64, device="cuda"))
    refiner.check()
    rng = np.random.default_rng(0)
    for _ in range(20):
        s, l, a = int(rng.integers(0, 64)), int(rng.integers(1, 7)), int(rng.integers(0, 3))
        h = 1e-2
        Pp, Pm = P.clone(), P.clone()
        Pp[s, l, a] += h
        Pm[s, l, a] -= h
        fp = refiner.forward(Pp, T, A, b, nr)[s].item()
        fm = refiner.forward(Pm, T, A, b, nr)[s].item()
        fd = (fp - fm) / (2 * h)
        g = dP[s, l, a].item()
        assert abs(fd - g) <= 2e-2 * max(1.0, abs(g), abs(fd)), (fd, g)
