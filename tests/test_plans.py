"""Host logic of the expansion planner, without a GPU (tx_describe_expansion_plan): the plan of
the Pt-shaped bench workload against the launch record of its ncu profile, and the limits every
plan must respect (shared memory per CTA, TMEM columns, the persistent kernel's conditions) over
a sweep of shapes and precisions."""
import itertools

import pytest

import paper_2401_04189_gb300 as P

MAX_DYN_SMEM = 227 * 1024          # opt-in dynamic shared memory per CTA (sm_100 family)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_04189_gb300 import build
    build.build()


def pad8(v):
    return (v + 7) // 8 * 8


def pad16(v):
    return (v + 15) // 16 * 16


def test_pt_shaped_bf16_plan():
    """96^3, rank 40, 40 terms, bf16: the persistent kernel (384 threads) with 2 planes per item,
    so 48 items per pair; four Y buffers of 80 TMEM columns and phi 2 x 96.  Form 1 gives the
    one-CTA-per-item kernel, form 2 the persistent kernel with stage 3 in bf16 (512 threads, one
    plane per item, phi double-buffered, three Y buffers of 48 columns)."""
    d = P.tx_describe_expansion_plan((96, 96, 96), (40, 40, 40), 40, "bf16")
    assert d["kernel"] == "persistent" and d["threads"] == 384
    assert (d["planes"], d["items_per_pair"]) == (2, 48)
    assert (d["ybuffers"], d["tmem_cols"]) == (4, 512)       # 4 x 80 Y columns + 2 x 96 phi columns
    assert (d["ksteps2"], d["ksteps3"]) == (3, 5)            # bf16 K = 16 per step (40 -> 48); tf32 K = 8
    assert d["stages2"] >= 3 and d["stages3"] >= 3            # the epilogue needs no staging buffers
    one = P.tx_describe_expansion_plan((96, 96, 96), (40, 40, 40), 40, "bf16", form=1)
    assert one["kernel"] == "per_item" and one["threads"] == 352
    b = P.tx_describe_expansion_plan((96, 96, 96), (40, 40, 40), 40, "bf16", form=2)
    assert b["kernel"] == "persistent_bf16" and b["threads"] == 512
    assert (b["planes"], b["items_per_pair"], b["ybuffers"]) == (1, 96, 3) and b["ksteps3"] == 3


def test_split_precisions_use_the_converter_kernel():
    for prec in ("tf32x3", "bf16x3"):
        d = P.tx_describe_expansion_plan((96, 96, 96), (40, 40, 40), 40, prec)
        assert d["kernel"] == "converter"
        # separate cross-product accumulators double the TMEM columns of Y and phi, and phi of a
        # slab (one plane: 96 rows of a 128-row tile, 96 columns) fits the converter warps'
        # float32 register accumulator (at most 128 columns per lane quadrant)
        assert d["planes"] == 1 and d["tmem_cols"] == 512
    assert P.tx_describe_expansion_plan((96, 96, 96), (40, 40, 40), 40, "fp32")["kernel"] == "float32"


def test_tio2_shaped_bf16_plan_takes_one_y_tile_per_item():
    """160^3, rank 64, 45 terms, bf16: a whole plane (two y tiles) would need 576 TMEM columns, so
    the persistent kernel takes one item per (pair, plane, y tile): phi 160 + four Y buffers of
    64 columns; the one-CTA-per-item form (form 1) falls back to the converter kernel."""
    d = P.tx_describe_expansion_plan((160, 160, 160), (64, 64, 64), 45, "bf16")
    # 160 full 128-row tiles, then the 32-row last tiles of four planes per item: 160 + 40
    assert d["kernel"] == "persistent" and d["planes"] == 1 and d["items_per_pair"] == 200
    assert d["tail_planes"] == 4
    assert d["ybuffers"] == 4 and d["tmem_cols"] == 512
    assert d["stages2"] >= 2 and d["stages3"] >= 2
    u = P.tx_describe_expansion_plan((160, 160, 160), (64, 64, 64), 45, "bf16", form=3)
    assert u["kernel"] == "persistent" and u["items_per_pair"] == 320 and u["tail_planes"] == 0
    # 150 rows: the last tile has 22 rows (24 with padding), five planes per item; 30 planes
    v = P.tx_describe_expansion_plan((30, 150, 160), (24, 64, 64), 12, "bf16")
    assert v["tail_planes"] == 5 and v["items_per_pair"] == 30 + 6
    assert P.tx_describe_expansion_plan((160, 160, 160), (64, 64, 64), 45, "bf16", form=1)["kernel"] == "converter"
    b = P.tx_describe_expansion_plan((160, 160, 160), (64, 64, 64), 45, "bf16", form=2)
    assert b["kernel"] == "persistent_bf16" and b["items_per_pair"] == 320


SIZES = [(16, 16, 16), (20, 27, 36), (32, 32, 32), (48, 64, 80), (64, 64, 64), (96, 96, 96), (112, 112, 112),
         (128, 128, 128), (160, 160, 160), (200, 200, 200), (256, 256, 256)]
RANKS = [1, 5, 16, 32, 40, 48, 64]


@pytest.mark.parametrize("prec", ["bf16", "tf32", "tf32x3", "bf16x3"])
def test_every_plan_respects_the_hardware_limits(prec):
    tf32 = prec.startswith("tf32")
    split = prec.endswith("x3")
    mk = 8 if tf32 else 16
    planned = 0
    for n, r, T, form in itertools.product(SIZES, RANKS, (1, 40), (0, 1, 2, 3, 4, 5)):
        rr = tuple(min(r, v) for v in n)
        try:
            d = P.tx_describe_expansion_plan(n, rr, T, prec, form)
        except P.TuckerExchangeError as e:
            assert e.status == -9, (n, rr, T, form, str(e))     # unsupported shape, never another error
            continue
        planned += 1
        key = (n, rr, T, form, d)
        assert 0 < d["smem_bytes"] <= MAX_DYN_SMEM, key
        assert d["tmem_cols"] in (32, 64, 128, 256, 512), key
        slabs = -(-n[0] // d["planes"])
        tp = d["tail_planes"]
        nz = d["z_parts"]
        if nz:                                  # split kernel, y/z items: plane x y tile x z part
            assert split and d["kernel"] == "converter" and d["planes"] == 1, key
            assert d["n3p"] == pad16(-(-n[2] // nz)) and (nz - 1) * d["n3p"] < n[2], key
            assert d["items_per_pair"] == n[0] * -(-n[1] // 128) * nz, key
            assert d["ksteps2"] == -(-rr[1] // mk) and d["ksteps3"] == -(-rr[2] // mk), key
            # TMEM: Y and phi with their cross-product accumulators; phi folds into 4 x 16 registers
            assert 2 * (pad16(rr[2]) + d["n3p"]) <= d["tmem_cols"] <= 512 and d["n3p"] <= 128, key
            continue
        if tp:                                  # packed last y tiles: full tiles, then tail groups
            nyf = -(-n[1] // 128)
            rows = n[1] - 128 * (nyf - 1)
            assert d["planes"] == 1 and tp == 128 // pad8(rows) >= 2 and form in (0, 2, 4, 5), key
            assert d["items_per_pair"] == n[0] * (nyf - 1) + -(-n[0] // tp), key
            yi = nyf
        else:
            yi = d["items_per_pair"] // slabs   # work items per slab: 1, or one per 128-row y tile
            assert d["planes"] >= 1 and d["items_per_pair"] == slabs * yi and yi in (1, -(-n[1] // 128)), key
        if yi > 1:
            assert d["kernel"] in ("persistent", "persistent_bf16", "persistent_bf16_tmem", "persistent_dual_issue") \
                and form in (0, 2, 3, 4, 5), key
        assert d["n3p"] == pad16(n[2]), key
        assert d["ksteps2"] == -(-rr[1] // mk), key
        assert d["stages2"] >= 1, key
        if split:
            assert d["kernel"] == "converter", key
            assert d["ksteps3"] == -(-rr[2] // mk), key
            assert 1 <= d["stages3"] <= 2, key     # the stage-3 operand ring
            continue
        if d["kernel"] == "converter":          # single-pass shapes no TMEM plan holds
            assert 1 <= d["stages3"] <= 2, key     # the stage-3 operand ring
            continue
        if d["kernel"] == "persistent_bf16":
            assert prec == "bf16" and form == 2 and d["threads"] == 512, key
            assert d["ksteps3"] == -(-rr[2] // 16) and d["ybuffers"] >= 2 and d["stages3"] >= 2, key
            assert d["planes"] <= (2 if yi > 1 else 4) and d["stages2"] <= 4, key
            continue
        if d["kernel"] == "persistent_bf16_tmem":
            # Y rounded to bf16 in TMEM by eight converter warps, two phi buffers, four epilogue warps
            assert prec == "bf16" and form == 4 and d["threads"] == 512, key
            assert d["ksteps3"] == -(-rr[2] // 16) and pad8(rr[2]) % 32 == 0, key
            assert d["ybuffers"] >= 2 and d["stages3"] >= 2 and d["planes"] <= 2, key
            continue
        assert d["ksteps3"] == -(-rr[2] // 8), key                # stage 3 is tf32 with A from TMEM
        assert d["ybuffers"] >= 2 and d["stages3"] >= 2, key
        if d["kernel"] == "persistent_dual_issue":
            # two stage-2 and two stage-3 MMA warps, two phi buffers read in place by eight warps
            assert prec == "bf16" and form == 5 and T >= 2 and d["threads"] == 448, key
            assert d["planes"] <= 2 and d["stages2"] <= 4, key
            tiles = d["planes"] * (1 if yi > 1 else -(-n[1] // 128))
            assert tiles <= 2 and d["ybuffers"] * pad8(rr[2]) * d["planes"] + 2 * tiles * d["n3p"] <= 512, key
            continue
        if d["kernel"] == "persistent":
            assert form in (0, 2, 3, 4, 5) and d["threads"] == 384, key
            assert d["planes"] <= 2 and d["stages2"] <= 4, key
            tiles = d["planes"] * (1 if yi > 1 else -(-n[1] // 128))
            assert tiles <= 2, key                                  # at most one phi tile per epilogue warp
            # an epilogue lane holds its row of phi (two tiles) or every other 32-column chunk (one)
            assert (d["n3p"] <= 96) if tiles == 2 else (32 * ((-(-d["n3p"] // 32) + 1) // 2) <= 96), key
        else:
            assert d["kernel"] == "per_item" and d["threads"] == 352, key
    assert planned > 50


def test_shapes_the_tensor_cores_cannot_take_are_refused():
    with pytest.raises(P.TuckerExchangeError) as ei:
        P.tx_describe_expansion_plan((12, 13, 15), (3, 4, 5), 3, "bf16")     # 15 floats: rows not 16-byte
    assert ei.value.status == -9
    P.tx_describe_expansion_plan((12, 13, 15), (3, 4, 5), 3, "fp32")
    with pytest.raises(P.TuckerExchangeError) as ei:
        P.tx_describe_expansion_plan((12, 13, 300), (3, 4, 5), 3, "fp32")    # float32 kernels: n3 <= 256
    assert ei.value.status == -9
    for bad, status in [(((1, 8, 8), (1, 1, 1), 3, "bf16", 0), -2), (((8, 8, 8), (9, 1, 1), 3, "bf16", 0), -2),
                        (((8, 8, 8), (2, 2, 2), 0, "bf16", 0), -1), (((8, 8, 8), (2, 2, 2), 3, "bf16", 6), -1)]:
        with pytest.raises(P.TuckerExchangeError) as ei:
            P.tx_describe_expansion_plan(*bad)
        assert ei.value.status == status, bad
