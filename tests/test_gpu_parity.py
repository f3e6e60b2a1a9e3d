"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs (float32 orbitals promoted to float64 on the oracle side)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from _helpers import E_TOL, W_TOL, _log, assert_close, elem_rel, log_energy, max_row_rel, rel, to_gpu

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16", "tf32", "tf32x3", "bf16x3"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def _P():
    import paper_2401_04189_gb300 as P
    return P


def ragged_system(n=(20, 27, 36), r=(5, 7, 9), T=7, n_orb=5, seed=3):
    """Different n and r per mode, none a multiple of a tile size (n3 a multiple of 4, as the
    tensor-core path needs 16-byte orbital rows)."""
    rng = np.random.default_rng(seed)
    Ls = [0.22 * (k - 1) / 2 for k in n]
    xs, ws = zip(*[W.uniform_grid(k, L) for k, L in zip(n, Ls)])
    cen = rng.uniform(-1.5, 1.5, size=(n_orb, 3, 3))
    exps = rng.uniform(0.4, 2.0, size=(n_orb, 3))
    coefs = rng.standard_normal(size=(n_orb, 3))
    psi = W.lowdin_orthonormalise(W.gaussian_sum_orbitals(xs, cen, exps, coefs), ws).astype(np.float32)
    U = W.density_hosvd_basis(psi, r)
    h = min(float(np.min(np.diff(v))) for v in xs)
    theta, mu, ferr = W.exp_sum_inverse_r(T, h, math.sqrt(sum((2 * L) ** 2 for L in Ls)))
    return W.System("ragged", list(xs), list(ws), U, theta, mu, psi, ferr)


def gpu_apply(s, prec, tgt=None, occ_idx=None, limit=None):
    P = _P()
    ctx = P.Context.from_system(s, precision=prec)
    if limit:
        ctx.set_workspace_limit(limit)
    occ = to_gpu(s.psi)
    if isinstance(tgt, str):
        out = P.tx_exchange_apply(ctx, occ)
    elif isinstance(tgt, slice):
        out = P.tx_exchange_apply(ctx, occ, occ[tgt])
    else:
        out = P.tx_exchange_apply(ctx, occ, to_gpu(tgt))
    ctx.check_device_error()          # a bounded device-side wait that gave up fails the test
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", PRECS)
def test_apply_small_config_matches_oracle(prec):
    s = W.config_small()
    S = O.Setup.from_system(s)
    ref = O.exchange_apply(s.psi, S)
    got = gpu_apply(s, prec, "self")
    assert_close(got, ref, prec, "small")
    assert max_row_rel(got, ref) < 2 * W_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_energy_small_config_matches_oracle(prec):
    P = _P()
    s = W.config_small()
    S = O.Setup.from_system(s)
    ref = O.exchange_energy(s.psi, S)
    ctx = P.Context.from_system(s, precision=prec)
    e = float(P.tx_exchange_energy(ctx, to_gpu(s.psi)).item())
    log_energy(prec, "small", e, ref)
    assert ref < 0
    assert abs(e - ref) / abs(ref) < E_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("targets", ["self", "subset", "general"])
def test_apply_ragged_shapes(prec, targets):
    s = ragged_system()
    S = O.Setup.from_system(s)
    if targets == "self":
        ref = O.exchange_apply(s.psi, S)
        got = gpu_apply(s, prec, "self")
    elif targets == "subset":
        ref = O.exchange_apply(s.psi, S, psi_tgt=s.psi[1:4])
        got = gpu_apply(s, prec, slice(1, 4))
    else:
        rng = np.random.default_rng(9)
        tgt = (s.psi[:3] * 0.7 + 0.2 * rng.standard_normal(s.psi[:3].shape) * np.abs(s.psi[:3]).max()).astype(np.float32)
        ref = O.exchange_apply(s.psi, S, psi_tgt=tgt)
        got = gpu_apply(s, prec, tgt)
    assert_close(got, ref, prec, f"ragged-{targets}")


@pytest.mark.parametrize("prec", PRECS)
def test_pair_batching_does_not_change_the_result(prec):
    s = ragged_system(n_orb=6)
    one = gpu_apply(s, prec, "self")
    many = gpu_apply(s, prec, "self", limit=1 << 20)     # forces one or two pairs per batch
    assert rel(many, one) < 1e-6


@pytest.mark.parametrize("prec", PRECS)
def test_single_orbital_single_term(prec):
    s = W.config_small(n=16, n_orb=1, rank=6, T=1, L=5.0)
    S = O.Setup.from_system(s)
    assert_close(gpu_apply(s, prec, "self"), O.exchange_apply(s.psi, S), prec, "single")


@pytest.mark.parametrize("prec", PRECS)
def test_full_rank_operator(prec):
    s = W.config_small(n=16, n_orb=3, rank=16, T=6, L=5.0, full_rank=True)
    S = O.Setup.from_system(s)
    assert_close(gpu_apply(s, prec, "self"), O.exchange_apply(s.psi, S), prec, "full-rank")


@pytest.mark.parametrize("prec", PRECS)
def test_energy_gradient_matches_oracle(prec):
    P = _P()
    s = ragged_system(n=(14, 17, 20), r=(5, 6, 7), T=5, n_orb=3)
    S = O.Setup.from_system(s)
    E_ref, g_ref = O.exchange_energy_grad(s.psi, S)
    ctx = P.Context.from_system(s, precision=prec)
    e, g = P.tx_exchange_energy_grad(ctx, to_gpu(s.psi))
    assert abs(float(e.item()) - E_ref) / abs(E_ref) < E_TOL[prec]
    assert_close(g.cpu().numpy(), g_ref, prec, "grad", scale=5)


@pytest.mark.parametrize("prec", PRECS)
def test_apply_vjp_matches_oracle(prec):
    P = _P()
    s = ragged_system(n=(14, 17, 20), r=(5, 6, 7), T=5, n_orb=3)
    S = O.Setup.from_system(s)
    rng = np.random.default_rng(4)
    tgt = (s.psi[:2] + 0.1 * s.psi[1:3]).astype(np.float32)
    cot = rng.standard_normal(tgt.shape).astype(np.float32)
    go_ref, gt_ref = O.exchange_apply_vjp(s.psi, tgt, cot, S)
    ctx = P.Context.from_system(s, precision=prec)
    go, gt = P.tx_exchange_apply_vjp(ctx, to_gpu(s.psi), to_gpu(tgt), to_gpu(cot))
    assert_close(go.cpu().numpy(), go_ref, prec, "vjp-occ", scale=5)
    assert_close(gt.cpu().numpy(), gt_ref, prec, "vjp-tgt", scale=5)


@pytest.mark.parametrize("prec", PRECS)
def test_pt_shaped_block_sampled_rows(prec):
    """Full Pt-shaped size (96^3, 64 orbitals, rank 40, 40 terms); the oracle computes two
    target rows against all 64 occupied orbitals."""
    s = W.config_pt()
    S = O.Setup.from_system(s)
    got = gpu_apply(s, prec, "self")
    for i in (0, 37):
        ref = O.exchange_apply(s.psi, S, psi_tgt=s.psi[i:i + 1])
        assert_close(got[i:i + 1], ref, prec, f"pt-row{i}")


def test_invalid_alignment_and_null_are_rejected():
    P = _P()
    import torch
    s = W.config_small(n=12, n_orb=2, rank=4, T=2, L=4.0)
    ctx = P.Context.from_system(s)
    occ = to_gpu(s.psi)
    buf = torch.zeros(occ.numel() + 1, dtype=torch.float32, device="cuda")
    mis = buf[1:].view(occ.shape)                      # 4-byte offset: not 16-byte aligned
    st = P.lib().tx_exchange_apply(ctx.handle, mis.data_ptr(), 2, None, 0, occ.data_ptr(), None)
    assert st == -10
    st = P.lib().tx_exchange_energy(ctx.handle, occ.data_ptr(), 2, None, None)
    assert st == -1


def test_outputs_overlapping_inputs_are_rejected():
    """An output block that shares memory with an input block is refused before any launch
    (TX_ERR_INVALID_ARG); an output right after the inputs is accepted and correct."""
    P = _P()
    import torch
    s = W.config_small(n=12, n_orb=2, rank=4, T=2, L=4.0)
    ctx = P.Context.from_system(s, precision="fp32")
    L = P.lib()
    buf = torch.zeros((3,) + tuple(s.psi.shape[1:]), dtype=torch.float32, device="cuda")
    buf[:2] = to_gpu(s.psi)
    e = torch.zeros((), dtype=torch.float64, device="cuda")
    occ, second, third = buf.data_ptr(), buf[1].data_ptr(), buf[2].data_ptr()
    assert L.tx_exchange_apply(ctx.handle, occ, 2, None, 0, occ, None) == -1
    assert L.tx_exchange_apply(ctx.handle, occ, 2, None, 0, second, None) == -1
    assert L.tx_exchange_apply(ctx.handle, occ, 1, third, 1, third, None) == -1      # out on the target
    assert L.tx_exchange_apply_energy(ctx.handle, occ, 2, second, e.data_ptr(), None) == -1
    assert L.tx_exchange_energy_grad(ctx.handle, occ, 2, second, e.data_ptr(), None) == -1
    assert L.tx_exchange_apply_vjp(ctx.handle, occ, 2, occ, 1, third, second, None, None) == -1
    assert L.tx_exchange_apply_static(ctx.handle, occ, 2, second, None) == -1
    assert L.tx_exchange_apply(ctx.handle, occ, 2, occ, 1, third, None) == 0         # adjacent: fine
    ctx.check_device_error()
    S = O.Setup.from_system(s)
    ref = O.exchange_apply(s.psi, S, psi_tgt=s.psi[0:1])
    assert rel(buf[2:3].cpu().numpy(), ref) < W_TOL["fp32"]


def test_empty_target_block_gives_empty_result():
    P = _P()
    import torch
    s = W.config_small(n=12, n_orb=2, rank=4, T=2, L=4.0)
    ctx = P.Context.from_system(s, precision="fp32")
    occ = to_gpu(s.psi)
    for tgt in (occ[:0], torch.empty((0, 12, 12, 12), dtype=torch.float32, device="cuda")):
        assert tuple(P.tx_exchange_apply(ctx, occ, tgt).shape) == (0, 12, 12, 12)
    ctx.check_device_error()


@pytest.mark.parametrize("prec", ["bf16", "tf32x3"])
def test_tensor_core_precisions_reject_unaligned_rows(prec):
    P = _P()
    s = ragged_system(n=(12, 13, 15), r=(3, 4, 5), T=3, n_orb=2)
    with pytest.raises(P.TuckerExchangeError) as ei:
        P.Context.from_system(s, precision=prec)
    assert ei.value.status == -9
    P.Context.from_system(s, precision="fp32")          # the float32 path takes any shape


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_accumulation_chunk_bounds_the_accumulator_error(prec):
    """The final contraction accumulates on the tensor core for `chunk` Gaussian terms before it
    is folded into the float32 register accumulator.  The default (a fold after every term) and
    an explicit chunk of 1 meet the precision's tolerance; longer chunks let the tensor core's
    truncating accumulator run longer and are not more accurate than a fold after every term."""
    P = _P()
    s = W.config_small()
    S = O.Setup.from_system(s)
    ref = O.exchange_apply(s.psi, S)
    errs = {}
    for ch in (0, 1, 7, 1000):
        ctx = P.Context.from_system(s, precision=prec)
        P.tx_set_accumulation_chunk(ctx, ch)
        got = P.tx_exchange_apply(ctx, to_gpu(s.psi)).cpu().numpy()
        ctx.check_device_error()
        errs[ch] = rel(got, ref)
        _log(dict(what=f"chunk{ch}", prec=prec, frob=errs[ch], elem=0.0))
        assert errs[ch] < (1 if ch in (0, 1) else 10) * W_TOL[prec], (ch, errs[ch])
    # the default is one term per chunk (W is summed over pairs in an unordered float32 order, so
    # two runs differ in the last bits)
    assert abs(errs[0] - errs[1]) <= 0.25 * errs[1]
    assert errs[1] <= errs[1000] * 1.02
    with pytest.raises(P.TuckerExchangeError):
        P.tx_set_accumulation_chunk(P.Context.from_system(s, precision=prec), -1)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("system", ["small", "ragged", "pt8"])
def test_expansion_forms_agree(prec, system):
    """The persistent expansion kernel (default where it applies) and the one-CTA-per-item
    kernel give the same apply and energy (to float32 summation order), and match the oracle;
    for bf16 the third form (stage 3 in bf16 as well) agrees with them to the bf16 tolerance."""
    P = _P()
    if system == "small":
        s = W.config_small()
    elif system == "ragged":
        s = ragged_system()
    else:
        s = W.config_pt(n_orb=8)
    S = O.Setup.from_system(s)
    outs, energies = [], []
    for form in ((0, 1, 2) if prec == "bf16" else (0, 1)):
        ctx = P.Context.from_system(s, precision=prec)
        P.tx_set_expansion_form(ctx, form)
        occ = to_gpu(s.psi)
        outs.append(P.tx_exchange_apply(ctx, occ).cpu().numpy())
        energies.append(float(P.tx_exchange_energy(ctx, occ).item()))
        ctx.check_device_error()
    assert rel(outs[0], outs[1]) < 1e-5
    assert abs(energies[0] - energies[1]) <= 1e-5 * abs(energies[1])
    if prec == "bf16":         # form 2 also rounds the stage-3 operand Y to bf16
        assert rel(outs[2], outs[0]) < W_TOL[prec]
        assert abs(energies[2] - energies[0]) <= E_TOL[prec] * abs(energies[0])
    if system != "pt8":
        ref = O.exchange_apply(s.psi, S)
        assert_close(outs[0], ref, prec, f"forms-{system}")
        e_ref = O.exchange_energy(s.psi, S)
        assert abs(energies[0] - e_ref) / abs(e_ref) < E_TOL[prec]
    else:
        ref = O.exchange_apply(s.psi, S, psi_tgt=s.psi[3:4])
        assert_close(outs[0][3:4], ref, prec, "forms-pt8")
    with pytest.raises(P.TuckerExchangeError):
        P.tx_set_expansion_form(P.Context.from_system(s, precision=prec), 6)


@pytest.mark.parametrize("rank,prec,kernel", [(64, "bf16", "persistent"), (64, "tf32", "persistent"),
                                              (48, "bf16", "per_item"), (48, "tf32", "per_item")])
def test_large_grid_two_y_tiles(prec, rank, kernel):
    """n = 160: two 128-row y tiles per plane.  At rank 64 (the TiO2-shaped workload) a whole
    plane's stage-2 output buffers (2 x 128 TMEM columns) and phi (2 x 160) exceed TMEM's 512
    columns: bf16 and TF32 run the persistent kernel with one work item per full y tile (phi 160
    columns, four 64-column Y buffers) and the 32-row last tiles of four planes packed into one
    item; at rank 48 the one-CTA-per-item kernel.  Apply and energy against the oracle."""
    P = _P()
    assert P.tx_describe_expansion_plan((160, 160, 160), (rank,) * 3, 6, prec)["kernel"] == kernel
    s = W.config_small(n=160, n_orb=2, rank=rank, T=6, L=16.0)
    S = O.Setup.from_system(s)
    ref = O.exchange_apply(s.psi, S)
    ctx = P.Context.from_system(s, precision=prec)
    occ = to_gpu(s.psi)
    got = P.tx_exchange_apply(ctx, occ).cpu().numpy()
    e = float(P.tx_exchange_energy(ctx, occ).item())
    ctx.check_device_error()
    assert_close(got, ref, prec, f"n160-r{rank}")
    e_ref = O.exchange_energy(s.psi, S)
    log_energy(prec, f"n160-r{rank}", e, e_ref)
    assert abs(e - e_ref) / abs(e_ref) < E_TOL[prec]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("n,r,tail", [((27, 150, 160), (24, 64, 64), 5), ((12, 160, 160), (8, 64, 64), 4)])
def test_packed_short_y_tiles_match_the_unpacked_kernel_and_the_oracle(prec, n, r, tail):
    """Planes of more than 128 rows whose last y tile is short: the persistent kernel packs the
    last tiles of `tail` planes into one 128-row item (each plane's stage-2 operand a zero-padded
    window of A_t2).  27 planes in groups of 5 leave a partial group of 2; 150 rows leave a
    22-row tail (two zero rows of padding per plane).  Apply and energy against the unpacked form
    (form 3: the same arithmetic per element, so float32 summation order only) and the oracle;
    for bf16 also form 4 (stage 3 in bf16 from TMEM) against the oracle and form 5 (two warps
    issuing each stage's MMAs, the same arithmetic) against form 0."""
    P = _P()
    d = P.tx_describe_expansion_plan(n, r, 6, prec)
    assert d["kernel"] == "persistent" and d["tail_planes"] == tail
    s = ragged_system(n=n, r=r, T=6, n_orb=3, seed=5)
    S = O.Setup.from_system(s)
    occ = to_gpu(s.psi)
    outs, energies = [], []
    forms = (0, 3, 4, 5) if prec == "bf16" else (0, 3)
    for form in forms:
        ctx = P.Context.from_system(s, precision=prec)
        P.tx_set_expansion_form(ctx, form)
        outs.append(P.tx_exchange_apply(ctx, occ).cpu().numpy())
        energies.append(float(P.tx_exchange_energy(ctx, occ).item()))
        ctx.check_device_error()
    assert rel(outs[0], outs[1]) < 1e-5
    assert elem_rel(outs[0], outs[1])[0] < 1e-5
    assert abs(energies[0] - energies[1]) <= 1e-5 * abs(energies[1])
    ref = O.exchange_apply(s.psi, S)
    assert_close(outs[0], ref, prec, f"packed-{n[0]}x{n[1]}")
    if prec == "bf16":
        # form 4: Y rounded to bf16 in TMEM, stage 3 in bf16 (packed tiles, two phi buffers)
        assert P.tx_describe_expansion_plan(n, r, 6, prec, 4)["kernel"] == "persistent_bf16_tmem"
        assert_close(outs[2], ref, prec, f"packed-{n[0]}x{n[1]}-bf16tmem")
        assert abs(energies[2] - energies[0]) <= E_TOL[prec] * abs(energies[0])
        # form 5: the same MMAs in the same term order, issued by two warps per stage
        assert P.tx_describe_expansion_plan(n, r, 6, prec, 5)["kernel"] == "persistent_dual_issue"
        assert rel(outs[3], outs[0]) < 1e-5 and elem_rel(outs[3], outs[0])[0] < 1e-5
        assert abs(energies[3] - energies[0]) <= 1e-5 * abs(energies[0])
    e_ref = O.exchange_energy(s.psi, S)
    log_energy(prec, f"packed-{n[0]}x{n[1]}", energies[0], e_ref)
    assert abs(energies[0] - e_ref) / abs(e_ref) < E_TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,r,items", [((5, 150, 160), (5, 64, 64), 20), ((4, 100, 200), (4, 40, 64), 8)])
def test_split_precisions_on_y_z_items_match_oracle(prec, n, r, items):
    """Planes too large for the split kernel's whole-slab plan (phi and its cross-product
    accumulator exceed TMEM, or the register accumulator): one CTA per (plane, 128-row y tile,
    z part).  150 rows leave a 22-row second tile; 200 columns split 112 + 88.  Apply and energy
    against the oracle at the split tolerances, elementwise."""
    P = _P()
    d = P.tx_describe_expansion_plan(n, r, 6, prec)
    assert d["kernel"] == "converter" and d["planes"] == 1 and d["items_per_pair"] == items
    s = ragged_system(n=n, r=r, T=6, n_orb=3, seed=9)
    S = O.Setup.from_system(s)
    ctx = P.Context.from_system(s, precision=prec)
    occ = to_gpu(s.psi)
    got = P.tx_exchange_apply(ctx, occ).cpu().numpy()
    e = float(P.tx_exchange_energy(ctx, occ).item())
    ctx.check_device_error()
    assert_close(got, O.exchange_apply(s.psi, S), prec, f"yz-{n[1]}x{n[2]}")
    e_ref = O.exchange_energy(s.psi, S)
    log_energy(prec, f"yz-{n[1]}x{n[2]}", e, e_ref)
    assert abs(e - e_ref) / abs(e_ref) < E_TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16"])
@pytest.mark.parametrize("order,points", [(1, 2), (1, 5), (3, 4), (3, 7)])
def test_finite_element_quadrature_matches_oracle(prec, order, points):
    """Finite-element quadrature of the 1-D convolutions (Lagrange elements of order 1 and 3,
    Gauss-Legendre points per element; Eqs. quadVal, discInteg) set up on the GPU against the
    oracle's; n - 1 = 15, 24, 27 holds whole elements of both orders.  Switching back to nodal
    quadrature gives the nodal result again."""
    P = _P()
    s = ragged_system(n=(16, 25, 28), r=(6, 8, 9), T=9, n_orb=5, seed=11)
    S_fe = O.Setup.from_system(s, quadrature=("fe", order, points))
    ref = O.exchange_apply(s.psi, S_fe)
    ctx = P.Context.from_system(s, precision=prec)
    occ = to_gpu(s.psi)
    ctx.set_quadrature(order, points)
    got = P.tx_exchange_apply(ctx, occ).cpu().numpy()
    ctx.check_device_error()
    assert_close(got, ref, prec, f"fe-p{order}-q{points}")
    # the nodal result differs from the element one (by 1e-2 here: well outside the float32 and
    # split tolerances, so those precisions tell the two apart), and comes back
    ref0 = O.exchange_apply(s.psi, O.Setup.from_system(s))
    assert rel(ref0, ref) > 100 * W_TOL["tf32x3"]
    ctx.set_quadrature(0)
    got0 = P.tx_exchange_apply(ctx, occ).cpu().numpy()
    assert_close(got0, ref0, prec, "fe-back-to-nodal")


@pytest.mark.parametrize("targets", ["self", "subset", "general"])
def test_per_pair_bases_match_oracle(targets):
    """Per-pair Tucker bases (sequentially truncated HOSVD of every pair density, Eq.
    TuckerDecompField) on ragged shapes against the oracle's.  The bases themselves are fixed
    only up to signs and rotations inside degenerate eigenspaces, so the potential (which
    depends on the projectors) is compared; float32 Jacobi eigenvectors (orthogonal to about
    1e-6) and float32 Gram matrices put the bound at 10x the float32 path's (measured 4e-6 to
    1.1e-5).  A bf16 context runs the same float32 kernels."""
    P = _P()
    s = ragged_system()
    S = O.Setup.from_system(s)
    occ = to_gpu(s.psi)
    rng = np.random.default_rng(9)
    tgt = (s.psi[:3] * 0.7 + 0.2 * rng.standard_normal(s.psi[:3].shape) * np.abs(s.psi[:3]).max()).astype(np.float32)
    for prec in ("fp32", "bf16"):
        ctx = P.Context.from_system(s, precision=prec)
        if targets == "self":
            ref = O.exchange_apply_sthosvd(s.psi, S, s.r)
            got = P.tx_exchange_apply_sthosvd(ctx, occ)
        elif targets == "subset":
            ref = O.exchange_apply_sthosvd(s.psi, S, s.r, psi_tgt=s.psi[1:4])
            got = P.tx_exchange_apply_sthosvd(ctx, occ, occ[1:4])
        else:
            ref = O.exchange_apply_sthosvd(s.psi, S, s.r, psi_tgt=tgt)
            got = P.tx_exchange_apply_sthosvd(ctx, occ, to_gpu(tgt))
        ctx.check_device_error()
        got = got.cpu().numpy()
        err, err_e = rel(got, ref), elem_rel(got, ref)[0]
        _log(dict(what=f"sthosvd-{targets}", prec=prec, frob=err, elem=err_e))
        assert err < 2e-5 and err_e < 4e-5, (err, err_e)
    # the shared basis gives a different operator at this rank
    assert rel(O.exchange_apply(s.psi, S, psi_tgt=None if targets == "self" else
                                (s.psi[1:4] if targets == "subset" else tgt)), ref) > 1e-3


def test_per_pair_bases_at_full_rank_are_exact():
    """At full rank every projector is the identity, so the result is unique whatever
    eigenvectors the solver returns; the float32 Jacobi rotations leave the eigenvector matrices
    orthogonal to about 1e-6 only, which puts the bound at 5x the float32 path's (measured
    5.5e-6)."""
    P = _P()
    s = ragged_system(n=(12, 14, 16), r=(12, 14, 16), T=5, n_orb=3, seed=8)
    S = O.Setup.from_system(s)
    ref = O.exchange_apply_sthosvd(s.psi, S, s.r)
    ctx = P.Context.from_system(s, precision="fp32")
    got = P.tx_exchange_apply_sthosvd(ctx, to_gpu(s.psi)).cpu().numpy()
    ctx.check_device_error()
    assert_close(got, ref, "fp32", "sthosvd-full-rank", scale=5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("targets", ["self", "subset", "general"])
def test_galerkin_apply_matches_oracle(prec, targets):
    """The two-sided projection (P^* C P) on ragged shapes: the float32 CUDA-core path in every
    precision of the context, against the oracle's two-sided operator; the exchange matrix of the
    occupied block is symmetric to float32 rounding at this truncated rank."""
    P = _P()
    s = ragged_system()
    S = O.Setup.from_system(s)
    ctx = P.Context.from_system(s, precision=prec)
    occ = to_gpu(s.psi)
    if targets == "self":
        ref = O.exchange_apply_galerkin(s.psi, S)
        got = P.tx_exchange_apply_galerkin(ctx, occ)
    elif targets == "subset":
        ref = O.exchange_apply_galerkin(s.psi, S, psi_tgt=s.psi[1:4])
        got = P.tx_exchange_apply_galerkin(ctx, occ, occ[1:4])
    else:
        rng = np.random.default_rng(9)
        tgt = (s.psi[:3] * 0.7 + 0.2 * rng.standard_normal(s.psi[:3].shape) * np.abs(s.psi[:3]).max()).astype(np.float32)
        ref = O.exchange_apply_galerkin(s.psi, S, psi_tgt=tgt)
        got = P.tx_exchange_apply_galerkin(ctx, occ, to_gpu(tgt))
    ctx.check_device_error()
    got = got.cpu().numpy()
    assert_close(got, ref, "fp32", f"galerkin-{targets}")
    # the one-sided operator differs here by far more than the tolerance
    assert rel(O.exchange_apply(s.psi, S, psi_tgt=None if targets == "self" else
                                (s.psi[1:4] if targets == "subset" else tgt)), ref) > 100 * W_TOL["fp32"]
    if targets == "self":
        w3 = S.w3[None]
        M = np.einsum("axyz,bxyz->ab", s.psi.astype(np.float64) * w3, got.astype(np.float64))
        assert np.max(np.abs(M - M.T)) < 2e-6 * np.max(np.abs(M))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_galerkin_energy_in_core_space_matches_oracle(prec):
    """E_x of the two-sided form, summed in core space, against the oracle's and against the
    grid energy 1/2 sum_i <psi_i, W_i>_w of the GPU's own two-sided apply."""
    P = _P()
    s = W.config_small()
    S = O.Setup.from_system(s)
    ctx = P.Context.from_system(s, precision=prec)
    occ = to_gpu(s.psi)
    e = float(P.tx_exchange_energy_galerkin(ctx, occ).item())
    ref = O.exchange_energy_galerkin(s.psi, S)
    log_energy(prec, "galerkin-core", e, ref)
    assert abs(e - ref) < E_TOL["fp32"] * abs(ref)
    Wg = P.tx_exchange_apply_galerkin(ctx, occ)
    e_grid = float(P.tx_exchange_energy_from_w(ctx, occ, Wg).item())
    assert abs(e_grid - ref) < E_TOL["fp32"] * abs(ref)
    assert e < 0


def test_finite_element_quadrature_rejects_bad_orders():
    P = _P()
    s = ragged_system(n=(16, 25, 28), r=(6, 8, 9), T=5, n_orb=3, seed=11)
    ctx = P.Context.from_system(s, precision="fp32")
    for order, points in ((2, 3), (9, 3), (-1, 3), (3, 0), (3, 65)):   # 15 is odd: no order-2 elements
        with pytest.raises(P.TuckerExchangeError):
            ctx.set_quadrature(order, points)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_sharded_apply_matches_oracle(prec):
    """exchange_apply_sharded over 1, 2 and 3 ranks: each rank's target slice against the
    oracle's rows for the same targets."""
    P = _P()
    from paper_2401_04189_gb300.sharding import exchange_apply_sharded
    s = ragged_system(n_orb=5)
    S = O.Setup.from_system(s)
    ref = O.exchange_apply(s.psi, S)
    ctx = P.Context.from_system(s, precision=prec)
    occ = to_gpu(s.psi)
    for world in (1, 2, 3):
        for rank in range(world):
            a, b, Wl = exchange_apply_sharded(ctx, occ, world, rank)
            ctx.check_device_error()
            assert Wl.shape[0] == b - a
            if b > a:
                assert_close(Wl.cpu().numpy(), ref[a:b], prec, "sharded")


@pytest.fixture(scope="module")
def diff_case():
    """The differentiation workload's grid, rank and terms (64^3 on [-10, 10]^3, rank 32, 35
    terms) with 8 of its 32 orbitals, so that the oracle's E_x and full gradient take seconds."""
    s = W.config_diff(n_orb=8)
    S = O.Setup.from_system(s)
    E_ref, g_ref = O.exchange_energy_grad(s.psi, S)
    return s, E_ref, g_ref


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_energy_gradient_differentiation_workload(prec, diff_case):
    """E_x and dE_x/dpsi against the oracle, directly and through the autograd wrapper."""
    P = _P()
    s, E_ref, g_ref = diff_case
    ctx = P.Context.from_system(s, precision=prec)
    psi = to_gpu(s.psi)
    e, g = P.tx_exchange_energy_grad(ctx, psi)
    ctx.check_device_error()
    assert abs(float(e.item()) - E_ref) / abs(E_ref) < E_TOL[prec]
    g = g.cpu().numpy()
    assert_close(g, g_ref, prec, "grad-diff", scale=5)
    x = psi.clone().requires_grad_(True)
    E = P.exchange_energy(ctx, x)
    E.backward()
    ctx.check_device_error()
    assert abs(float(E.detach().item()) - E_ref) / abs(E_ref) < E_TOL[prec]
    assert rel(x.grad.cpu().numpy(), g) < 1e-5


@pytest.fixture(scope="module")
def tio2_case():
    """The TiO2-shaped workload's grid, rank and Gaussian sum (160^3 on [-16,16]^3, rank 64, 45
    terms; orbitals as in that workload: Gaussian sums over 16 of 240 rutile-like centres) with 8
    orbitals, so that the oracle's rows take seconds."""
    s = W.make_system("tio2", 160, 16.0, 8, 64, 45, 4, W.rutile_cluster(240), 2, (0.2, 3.0),
                      centres_per_orbital=16)
    S = O.Setup.from_system(s)
    refs = {i: O.exchange_apply(s.psi, S, psi_tgt=s.psi[i:i + 1]) for i in (0, 5)}
    return s, refs


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32", "tf32x3"])
def test_tio2_shaped_block_45_terms(prec, tio2_case):
    """Full target rows of the TiO2-shaped grid at all 45 terms against the oracle (the largest
    configuration's grid, rank and terms; the bench runs its full 256 x 1842 block).  The split
    precision runs y/z items there (one 128-row y tile and half the z columns per CTA)."""
    s, refs = tio2_case
    got = gpu_apply(s, prec, "self")
    for i, ref in refs.items():
        assert_close(got[i:i + 1], ref, prec, f"tio2-row{i}")


@pytest.fixture(scope="module")
def diff_full():
    """The differentiation workload in full (64^3 on [-10,10]^3, all 32 orbitals, rank 32, 35
    terms) with the oracle's gradient rows 0 and 17, each computed on its own:
    dE/dpsi_k = w W_k - sum_j psi_j L^T(w psi_k psi_j)."""
    s = W.config_diff()
    S = O.Setup.from_system(s)
    occ = s.psi.astype(np.float64)
    rows = {}
    for k in (0, 17):
        Wk = O.exchange_apply(occ, S, psi_tgt=occ[k:k + 1])[0]
        g = S.w3 * Wk
        for j in range(occ.shape[0]):
            g = g - occ[j] * O.apply_LT(S.w3 * occ[k] * occ[j], S)
        rows[k] = g
    return s, rows


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_differentiation_workload_all_orbitals(prec, diff_full):
    """All 32 orbitals of the differentiation workload in the split-precision form (and float32):
    gradient rows against the oracle's, and the gradient against central differences of the
    GPU's own energy along 20 seeded unit directions v = cos(a) g/|g| + sin(a) z/|z| (z random,
    a spread over [0, pi/2]).  The error is measured against |g|, the scale of any directional
    derivative: along a nearly orthogonal direction the derivative itself is close to zero and
    the float32 energy's rounding (about 1e-7 |E| / 2h) dominates.  E is a quartic polynomial in
    psi, so a step of 5e-2 on |psi| ~ 30 leaves a truncation error far below the bound."""
    import torch
    P = _P()
    s, rows = diff_full
    ctx = P.Context.from_system(s, precision=prec)
    psi = to_gpu(s.psi)
    e, g = P.tx_exchange_energy_grad(ctx, psi)
    ctx.check_device_error()
    gh = g.cpu().numpy().astype(np.float64)
    for k, ref in rows.items():
        assert_close(gh[k:k + 1].astype(np.float32), ref[None], prec, f"grad-diff-full-row{k}", scale=5)
    gn = float(np.linalg.norm(gh))
    ghat = gh / gn
    rng = np.random.default_rng(3)
    h = 5e-2
    errs = []
    for a in np.linspace(0.0, np.pi / 2, 20):
        z = rng.standard_normal(s.psi.shape)
        z -= np.sum(z * ghat) * ghat
        v = np.cos(a) * ghat + np.sin(a) * z / np.linalg.norm(z)
        vt = to_gpu(v)
        ep = float(P.tx_exchange_energy(ctx, psi + h * vt).item())
        em = float(P.tx_exchange_energy(ctx, psi - h * vt).item())
        fd = (ep - em) / (2 * h)
        dd = float(np.sum(gh * v))
        errs.append(abs(fd - dd) / gn)
    _log(dict(what="fd-diff-full", prec=prec, frob=max(errs), elem=0.0))
    assert max(errs) < 1e-3, errs
    torch.cuda.synchronize()
