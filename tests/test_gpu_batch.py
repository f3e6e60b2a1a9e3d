"""Batched application over uneven systems through one plan: results equal the individual
calls, the captured CUDA graph replays them, the autotuner writes its table, and a system of
the batch matches the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import W_TOL, assert_close, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def uneven_systems(shrink=True):
    """The shapes of the uneven batch (n, rank and term count drawn per system); the orbital
    counts are cut to at most 10 so the test stays short."""
    specs = W.batched_system_specs(count=6, base_seed=100)
    out = []
    for sp in specs:
        sp = dict(sp)
        if shrink:
            sp["n_orb"] = min(sp["n_orb"], 10)
        out.append(W.config_batched_system(sp))
    return out


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_batch_equals_individual_calls_and_graph_replay(prec, tmp_path):
    import torch
    import paper_2401_04189_gb300 as P
    systems = uneven_systems()
    ctxs = [P.Context.from_system(s, precision=prec) for s in systems]
    psis = [to_gpu(s.psi) for s in systems]
    ref_W = []
    ref_E = []
    for c, p in zip(ctxs, psis):
        w, e = P.tx_exchange_apply_energy(c, p)
        ref_W.append(w.cpu().numpy())
        ref_E.append(float(e.item()))
    table = tmp_path / "tune.txt"
    plan = P.BatchPlan([dict(ctx=c, psi_occ=p, energy=True) for c, p in zip(ctxs, psis)], tune_table=table,
                       autotune=True)
    assert table.exists() and len(table.read_text().splitlines()) >= 1
    for i in range(len(systems)):
        bx, ns = plan.item_plan(i)
        assert bx >= 1 and 1 <= ns <= 6
    for o in plan.outputs():
        o.zero_()
    plan.launch()
    torch.cuda.synchronize()
    for c in ctxs:
        c.check_device_error()
    for k in range(len(systems)):
        assert rel(plan.outputs()[k].cpu().numpy(), ref_W[k]) < 1e-5
        assert abs(plan.energies()[k].item() - ref_E[k]) < 1e-5 * abs(ref_E[k])
    # one CUDA graph holding every system, replayed
    s = torch.cuda.Stream()
    plan.capture(s)
    for o in plan.outputs():
        o.fill_(123.0)
    plan.replay(s)
    s.synchronize()
    for k in range(len(systems)):
        assert rel(plan.outputs()[k].cpu().numpy(), ref_W[k]) < 1e-5
    # a second plan reads the table instead of timing again
    before = table.read_text()
    plan2 = P.BatchPlan([dict(ctx=c, psi_occ=p) for c, p in zip(ctxs, psis)], tune_table=table, autotune=True)
    assert table.read_text() == before
    plan2.destroy()
    plan.destroy()


@pytest.mark.parametrize("prec", ["bf16", "tf32x3"])
def test_batch_systems_match_oracle(prec):
    """Every system of an uneven batch (six shapes of the batched configuration, up to 10
    orbitals each) against the oracle: whole systems (all targets) where n <= 64, two sampled
    target rows against all orbitals elsewhere; elementwise bounds of the precision."""
    import torch
    import paper_2401_04189_gb300 as P
    systems = uneven_systems()
    ctxs = [P.Context.from_system(s, precision=prec) for s in systems]
    psis = [to_gpu(s.psi) for s in systems]
    plan = P.BatchPlan([dict(ctx=c, psi_occ=p) for c, p in zip(ctxs, psis)])
    plan.launch()
    torch.cuda.synchronize()
    for c in ctxs:
        c.check_device_error()
    whole = 0
    for k, s in enumerate(systems):
        S = O.Setup.from_system(s)
        got = plan.outputs()[k].cpu().numpy()
        if s.n[0] <= 64:
            whole += 1
            ref = O.exchange_apply(s.psi, S)
            assert_close(got, ref, prec, f"batch-{k}-whole")
        else:
            rows = [0, len(s.psi) - 1]
            ref = O.exchange_apply(s.psi, S, psi_tgt=s.psi[rows])
            assert_close(got[rows], ref, prec, f"batch-{k}-rows")
    assert whole >= 1
    plan.destroy()


def test_forced_tile_plans_agree():
    import paper_2401_04189_gb300 as P
    s = W.config_small(n=48, n_orb=4, rank=20, T=8, L=6.0)
    ctx = P.Context.from_system(s, precision="bf16")
    psi = to_gpu(s.psi)
    base = P.tx_exchange_apply(ctx, psi).cpu().numpy()
    tried = 0
    for bx in (1, 2, 3, 5, 8, 13):
        for ns in (1, 2, 3, 4, 5, 6):
            try:
                P.tx_set_tile_plan(ctx, bx, ns)
            except P.TuckerExchangeError as e:
                assert e.status == -9
                continue
            tried += 1
            got = P.tx_exchange_apply(ctx, psi).cpu().numpy()
            assert rel(got, base) < 1e-5, (bx, ns)
    assert tried >= 3
    P.tx_set_tile_plan(ctx, 0, 0)
