"""Checkpoint / resume: a run stopped after its first half (with mid-circuit
measurements behind it) and resumed in a fresh context from the saved state,
the seed and the draw ordinal gives the same outcomes and state as the run
that never stopped, and as the oracle (the draw of the k-th measurement
depends only on (seed, k))."""
import numpy as np
import pytest

import oracle
from paper_2310_17739_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
qs = pytest.importorskip("paper_2310_17739_gb300.qsim")


@pytest.mark.parametrize("dtype,n,cfg", [("c128", 12, dict(fusion=1)), ("c64", 16, dict(fusion=2, tile_bits=12)),
                                         ("c128", 16, dict(fusion=2))])
def test_resume_from_state_seed_and_draw_ordinal(dtype, n, cfg):
    c = W.ucc_circuit(n, seed=300 + n, n_gadgets=None, w_lo=2, w_hi=6, theta="uniform", target_gates=6000,
                      n_meas=8)
    g = c.gates
    is_event = np.isin(g["op"], [W.OP["MEASURE"], W.OP["RESET"]])
    cut = int(np.flatnonzero(is_event)[3]) + 1        # after the 4th measurement
    seed = 41
    whole = qs.Sim(n, dtype, seed=seed, config=cfg)
    whole.apply(g)
    assert whole.sync() == 0
    out_whole, _ = whole.outcomes()
    # first half, checkpoint
    a = qs.Sim(n, dtype, seed=seed, config=cfg)
    a.apply(g[:cut])
    assert a.sync() == 0
    saved, k = a.state(), a.draw_ordinal()
    out_a, _ = a.outcomes()
    assert k == 4 == len(out_a)
    a.close()
    # resume in a fresh context
    b = qs.Sim(n, dtype, seed=seed, config=cfg)
    assert b.draw_ordinal() == 0
    b.set_state(saved)
    b.set_draw_ordinal(k)
    b.apply(g[cut:])
    assert b.sync() == 0
    out_b, _ = b.outcomes()
    assert b.draw_ordinal() == len(out_whole)
    assert np.array_equal(np.concatenate([out_a, out_b]), out_whole)
    got = b.state()
    # the resumed run is the same computation from the same state (its program
    # is compiled apart, so rounding may differ by an end-of-chunk frame flush)
    if dtype == "c128":
        assert np.abs(got - whole.state()).max() <= 1e-12
    else:
        assert 1 - H.fidelity(whole.state(), got) <= 1e-9
    ref = oracle.basis_state(n)
    r = oracle.run(ref, n, g, seed=seed)
    assert np.array_equal(r.outcomes, out_whole)
    if dtype == "c128":
        assert np.abs(got - ref).max() <= 1e-10
    else:
        assert 1 - H.fidelity(ref, got) <= 1e-5
    b.close()
    whole.close()
