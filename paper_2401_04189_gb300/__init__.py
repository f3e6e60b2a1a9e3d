"""GB300-native Tucker-tensor Fock exchange (arXiv 2401.04189 hot path).

The compute path is libtuxc.so (hand-written CUDA for sm_103a behind a C ABI declared in
include/tuxc.h).  This package is its thin Python binding plus torch.autograd wrappers.
"""
from ._lib import (  # noqa: F401
    Context, Precision, TuckerExchangeError, lib, tx_tucker_setup, tx_exchange_apply,
    tx_exchange_energy, tx_exchange_energy_grad, tx_exchange_apply_vjp, tx_launch_count,
    tx_reset_launch_count, tx_exchange_apply_energy, tx_profile_enable, tx_profile_reset,
    tx_profile_read, tx_selftest_gemm, BatchPlan, tx_set_tile_plan, tx_set_accumulation_chunk, tx_set_expansion_form, tx_describe_expansion_plan, EXPORTED, LIB_PATH,
    tx_exchange_energy_from_w, tx_selftest_wait, tx_ace_projectors, tx_ace_apply,
    tx_exchange_apply_galerkin, tx_exchange_energy_galerkin, Transfer, tx_exchange_apply_sthosvd,
)
TENSOR_CORE_PRECISIONS = ("bf16", "tf32", "tf32x3", "bf16x3")
DEFAULT_BENCH_PRECISION = "bf16"

from .autograd import ExchangeApply, ExchangeEnergy, exchange_apply, exchange_energy  # noqa: F401
