"""Precision form: the halves (H xi and A p products) on the tensor cores
(tcgen05.mma, TF32 or BF16 inputs, FP32 accumulation in tensor memory); every
margin inside its rounding band is re-checked in FP64, so masks, edge sets and
paths must still equal the FP64 oracle exactly.  The cost error against FP64
is reported (bounded loosely in tests/parity.py)."""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


@pytest.mark.parametrize("arith", ["tf32", "bf16"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tensor_core_form_bits_equal_fp64(arith, seed):
    prob = synth.double_integrator_2d(seed)
    pl = P.Planner.for_problem(prob, arith=arith, input="f64")
    dp = P.to_device(prob, input="f64")
    g = pl.build_edges(dp)
    info = pl.info()
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    st = parity.compare_full(g.to_numpy(), csr, prob.N, prob.nT, arith)
    gw = g.to_numpy()["w"]
    rel = np.abs(gw - csr["w"]) / csr["w"]
    print(f"{arith} seed {seed}: rechecks {info['rechecks']} of {info['checks']} checks "
          f"({100.0 * info['rechecks'] / max(1, info['checks']):.2f}%), cost rel err max {rel.max():.2e} "
          f"median {np.median(rel):.2e}")
    r = pl.search(dp, g)
    orc = oracle.search(op, csr, prob.start_pos, prob.goal_pos)
    parity.compare_search(r, orc, csr, arith)


@pytest.mark.parametrize("arith", ["tf32", "bf16"])
def test_tensor_core_form_minimal_degree_and_batched(arith):
    probs = [synth.double_integrator_2d(s, N=300, K=5, nT=6, degree=3) for s in (4, 5, 6)]
    pl = P.Planner.for_problem(probs[0], arith=arith, input="f64")
    dps = [P.to_device(p, input="f64") for p in probs]
    graphs = pl.build_batched(dps)
    for p, g in zip(probs, graphs):
        csr = oracle.OracleProblem(p).csr(with_detail=True)
        parity.compare_full(g.to_numpy(), csr, p.N, p.nT, arith)


def test_tensor_core_form_rejects_3d():
    with pytest.raises(P.PlanError):
        P.Planner(3, 3, 7, [3, 6, 30], arith="tf32", input="f32")
