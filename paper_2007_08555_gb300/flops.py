"""Algorithmic floating-point work of the evaluation path (for roofline fractions).

Counts what the method itself requires per unit, in the symmetric storage the kernels use,
counting an FMA as 2 flops and ignoring index arithmetic:

per neighbour pair, forward (moments kernel):
  geometry   |r| from r_ij: 5 (3 mul/add + sqrt counted as 1)
  radial     x = (2r - R_min - R_cut)/(R_cut - R_min): 3; Chebyshev recurrence (N_Q - 2) * 3;
             f_mu = sum_b c T_b: 2 N_mu N_Q; times (R_cut - r)^2: N_mu + 2
  monomials  one multiply per distinct monomial of degree >= 1
  moments    2 C  (one FMA per moment component)
per neighbour pair, adjoint (pair-gradient kernel):
  the geometry and radial terms again, with derivatives: + (N_Q - 2) * 5 + 2 N_mu N_Q + 4 N_mu
  monomials of the value and its gradient
  P_mu = sum adj mono, alpha_m = sum adj f: 4 C; s = sum df P: 2 N_mu; gradient terms
  2 per non-zero exponent; final r-hat scaling 7
per atom (contraction kernel): forward program 2 flops per op, adjoint 4 flops per op, site energy 2 m
per pair (gather kernel): force 6, virial 18
"""

from __future__ import annotations

from . import codegen


def counts(lev_max: int, n_radial: int):
    prog = codegen.build_program(lev_max)
    C = len(prog.comp_list)
    monos = sorted({m for _, m in prog.comp_list if m != (0, 0, 0)})
    grad_monos = set(monos)
    for m in monos:
        for k in range(3):
            if m[k] > 0:
                mm = list(m)
                mm[k] -= 1
                if tuple(mm) != (0, 0, 0):
                    grad_monos.add(tuple(mm))
    nmu = prog.n_mu
    NQ = n_radial
    radial_f = 3 + max(NQ - 2, 0) * 3 + 2 * nmu * NQ + nmu + 2
    radial_fd = radial_f + max(NQ - 2, 0) * 5 + 2 * nmu * NQ + 4 * nmu
    n_grad_terms = sum(sum(1 for k in range(3) if m[k] > 0) for m in monos)
    pair_fwd = 5 + radial_f + len(monos) + 2 * C
    pair_adj = 5 + radial_fd + len(grad_monos) + 4 * C + 2 * nmu + 2 * n_grad_terms + 7
    ops = len(prog.ops)
    atom_contract = 2 * ops + 4 * ops + 2 * prog.basis.m
    pair_gather = 6 + 18
    return {"C": C, "m": prog.basis.m, "ops": ops, "pair_moments": pair_fwd, "pair_adjoint": pair_adj,
            "atom_contract": atom_contract, "pair_gather": pair_gather}


def per_evaluation(lev_max: int, n_radial: int, n_atoms: int, n_pairs: int):
    """Flops of each kernel phase for one evaluation with the given atom and pair counts."""
    c = counts(lev_max, n_radial)
    return {"moments": c["pair_moments"] * n_pairs, "contract": c["atom_contract"] * n_atoms,
            "pairgrad": c["pair_adjoint"] * n_pairs, "gather": c["pair_gather"] * n_pairs}


def neighbor_bytes(n_atoms: int, n_pairs: int, real_bytes: int = 4) -> int:
    """Algorithmic DRAM bytes of one neighbour search (Eq. 1): per atom its position (3 doubles) and
    species read and its neighbour count written (32 B); per pair the neighbour index and r_ij in the
    path's precision written (4 + 3 real_bytes: 16 B on the float path)."""
    return 32 * n_atoms + (4 + 3 * real_bytes) * n_pairs


def fp32_peak_tflops(n_sm: int, clock_mhz: float) -> float:
    """FP32 FMA peak from unit counts: 128 lanes per SM, 2 flops per FMA, at the given SM clock
    (context for the measured figure of mtp_fp32_peak)."""
    return n_sm * 128 * 2 * clock_mhz * 1e6 / 1e12


def fp64_peak_tflops_nominal() -> float:
    """GB300 FP64 (nominal figure for context only)."""
    return 1.25
