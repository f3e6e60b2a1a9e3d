"""torch.autograd wrappers: the forward and the hand-written adjoint both run in libtuxc.so.

ExchangeEnergy:  E_x(psi) with dE/dpsi from tx_exchange_energy_grad (pair potentials are
                 recomputed in the backward call, not stored).
ExchangeApply:   W = K(psi_occ) psi_tgt with the VJP from tx_exchange_apply_vjp.
"""
from __future__ import annotations

import torch

from ._lib import Context, tx_exchange_apply, tx_exchange_apply_vjp, tx_exchange_energy, tx_exchange_energy_grad


class ExchangeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx: Context, psi):
        psi = psi.contiguous()
        fctx.tx = ctx
        fctx.save_for_backward(psi)
        return tx_exchange_energy(ctx, psi)

    @staticmethod
    def backward(fctx, gE):
        (psi,) = fctx.saved_tensors
        _, g = tx_exchange_energy_grad(fctx.tx, psi)
        return None, g * gE.to(g.dtype)


class ExchangeApply(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx: Context, psi_occ, psi_tgt):
        psi_occ = psi_occ.contiguous()
        psi_tgt = psi_tgt.contiguous()
        fctx.tx = ctx
        fctx.save_for_backward(psi_occ, psi_tgt)
        return tx_exchange_apply(ctx, psi_occ, psi_tgt)

    @staticmethod
    def backward(fctx, gW):
        psi_occ, psi_tgt = fctx.saved_tensors
        g_occ, g_tgt = tx_exchange_apply_vjp(fctx.tx, psi_occ, psi_tgt, gW.contiguous(),
                                             need_occ=fctx.needs_input_grad[1], need_tgt=fctx.needs_input_grad[2])
        return None, g_occ, g_tgt


def exchange_energy(ctx: Context, psi):
    return ExchangeEnergy.apply(ctx, psi)


def exchange_apply(ctx: Context, psi_occ, psi_tgt):
    return ExchangeApply.apply(ctx, psi_occ, psi_tgt)
