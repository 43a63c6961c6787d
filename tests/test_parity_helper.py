"""CPU checks of the parity comparison itself: the oracle matches itself, and
planted differences (a flipped mask bit, a weight off by more than the bar, a
missing edge, a wrong best duration) are each caught."""
import copy

import numpy as np
import pytest

import oracle
import parity
from paper_2411_13507_gb300 import synth


@pytest.fixture(scope="module")
def ref():
    prob = synth.double_integrator_2d(2, N=200, K=6)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    gpu = {"row_off": csr["row_off"], "col": csr["col"].copy(), "w": csr["w"].copy(), "t": csr["t"].copy(),
           "mask": csr["mask"].copy()}
    return prob, csr, gpu


def test_self_parity(ref):
    prob, csr, gpu = ref
    st = parity.compare_full(gpu, csr, prob.N, prob.nT, "f64")
    assert st["edges"] == len(csr["col"]) and st["tidx_checked"] > 0


@pytest.mark.parametrize("kind", ["mask", "weight", "col", "tidx"])
def test_planted_difference_caught(ref, kind):
    prob, csr, gpu = ref
    g = copy.deepcopy(gpu)
    k = len(g["col"]) // 2
    if kind == "mask":
        g["mask"][k] ^= np.uint32(1 << 7)
    elif kind == "weight":
        g["w"][k] *= 1 + 1e-7
    elif kind == "col":
        g["col"][k] += 1
    else:
        # a best duration with a clearly better alternative feasible duration
        e = csr["all"]
        keep = e["mask"] != 0
        costs, mask, t = e["costs"][keep], e["mask"][keep], e["t"][keep]
        for q in range(len(t)):
            alts = [s for s in range(prob.nT) if (int(mask[q]) >> s) & 1 and s != t[q]]
            if alts and all(costs[q, s] > costs[q, t[q]] * 1.01 for s in alts):
                g["t"][q] = alts[0]
                break
    with pytest.raises(AssertionError):
        parity.compare_full(g, csr, prob.N, prob.nT, "f64")
