"""Batched ensembles of 2-D Allen-Cahn instances (uneven sizes, per-instance
W, kappa, L): every stepping mode against the FP64 oracle, bitwise agreement
between the modes and before/after autotuning, and the bounded-barrier
failure path."""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu


def _pf():
    import paper_2601_06079_gb300 as pf
    return pf


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


SHAPES = [(64, 64), (37, 100), (128, 128), (91, 37), (130, 256), (4, 5)]


def make(shapes, seed=1):
    pf = _pf()
    e = pf.Ensemble(shapes)
    inst = G.batched_instances(seed, count=len(shapes))
    params = [dict(W=p["W"], kappa=p["kappa"], L=p["L"], dt=0.01) for p in inst]
    e.set_params(params)
    fields = [G.ac_initial(seed + i, s) for i, s in enumerate(shapes)]
    return e, params, fields


@pytest.mark.parametrize("mode", ["persistent", "per_step", "plain"])
def test_modes_match_oracle(mode):
    e, params, fields = make(SHAPES)
    st = e.pack(fields)
    e.step(st, 30, mode)
    torch.cuda.synchronize()
    for f, p, out in zip(fields, params, e.unpack(st)):
        ref = O.Problem(f.shape, W=p["W"], kappa=p["kappa"], mob=p["L"]).ac_explicit(f, 0.01, 30)
        assert rel(out.cpu().numpy(), ref) <= 1e-5


def test_modes_agree_bitwise_and_tuning_keeps_results():
    e, params, fields = make(SHAPES, seed=3)
    outs = {}
    for mode in ("plain", "per_step", "persistent"):
        st = e.pack(fields)
        e.step(st, 17, mode)
        outs[mode] = st.clone()
    assert torch.equal(outs["plain"], outs["per_step"])
    assert torch.equal(outs["plain"], outs["persistent"])
    ty, info = e.tune(reps=3)
    assert set(ty) <= {6, 12, 24}
    assert set(info["l2"]) <= set(e.L2_POLICIES)
    assert len(info["uniform_us"]) == 9 and all(u > 0 for u in info["uniform_us"].values())
    # the choice is never slower than the best single candidate by more than noise
    assert info["tuned_us"] <= min(info["uniform_us"].values()) * 1.0001
    assert all(u > 0 for row in info["trials_us"] for u in row.values())
    st = e.pack(fields)
    e.step(st, 17, "persistent")
    assert torch.equal(st, outs["plain"])
    # every schedule (band height x L2 policy, mixed across instances) is
    # bitwise equal to the plain form in both batched modes
    n = len(SHAPES)
    cands = e.candidates()
    for k in range(len(cands)):
        sched = [cands[(k + i) % len(cands)] for i in range(n)]
        e.set_schedule([c[0] for c in sched], [c[1] for c in sched])
        for mode in ("per_step", "persistent"):
            st = e.pack(fields)
            e.step(st, 17, mode)
            assert torch.equal(st, outs["plain"]), (k, mode)


def test_schedule_setter_rejects_bad_values():
    pf = _pf()
    e, _, _ = make(SHAPES, seed=4)
    with pytest.raises(pf.PFError):
        e.set_schedule(ty=[7] * len(SHAPES))
    with pytest.raises(ValueError):
        e.set_schedule(l2=["keep"] * len(SHAPES))
    assert pf._lib.pf_set_ensemble_schedule(e._ctx, None, [3] * len(SHAPES)) != 0


def test_256_instance_ensemble_1000_steps():
    pf = _pf()
    inst = G.batched_instances(1, count=256)
    shapes = [(p["n"], p["n"]) for p in inst]
    e = pf.Ensemble(shapes)
    params = [dict(W=p["W"], kappa=p["kappa"], L=p["L"], dt=0.01) for p in inst]
    e.set_params(params)
    e.tune(reps=3)
    fields = [G.ac_initial(100 + i, s) for i, s in enumerate(shapes)]
    st = e.pack(fields)
    e.step(st, 1000, "persistent")
    out = e.unpack(st)
    # the first instance of every size class against the oracle, 1000 steps
    O.set_threads(0)
    checked = set()
    for i, s in enumerate(shapes):
        if s[0] in checked:
            continue
        p = params[i]
        ref = O.Problem(s, W=p["W"], kappa=p["kappa"], mob=p["L"]).ac_explicit(
            fields[i], 0.01, 1000)
        assert rel(out[i].cpu().numpy(), ref) <= 1e-5, (i, s)
        checked.add(s[0])
    assert checked == {128, 256, 384, 512}
    st2 = e.pack(fields)
    e.step(st2, 1000, "per_step")
    assert torch.equal(st, st2)


def test_bounded_barrier_reports_timeout_and_context_survives():
    pf = _pf()
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert pf.pf_barrier_selftest(scratch.data_ptr(), 20_000_000, 0, s) == pf._lib.PF_OK
    assert pf.pf_barrier_selftest(scratch.data_ptr(), 2_000_000, 1, s) == pf._lib.PF_ERR_TIMEOUT
    x = torch.ones(8, device="cuda") * 2
    assert float(x.sum()) == 16.0  # the context still works
