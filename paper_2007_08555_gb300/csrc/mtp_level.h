// Per-level registry: generated tables and kernel launchers of one lev_max.
#pragma once
#include <cuda_runtime.h>
#include "mtp_common.cuh"

namespace mtp {

struct LevelOps {
    int L, C, V, M, NMU, NUMAX;
    const int* level_table;
    int level_table_len;
    const int* basis_value;        // [M] value index of each basis function
    const unsigned long long* fwd_ops;  // [rows][32] packed ops, see codegen.py
    const int* fwd_layer_end;
    int fwd_rows, fwd_layers;
    const unsigned long long* adj_ops;
    const int* adj_layer_end;
    int adj_rows, adj_layers;
    const float* weights;               // weight table indexed by the packed ops
    int n_weights;
    int program_ops;
    int flop_pair_moments, flop_pair_adjoint, flop_atom_program;
    int contract_parts, contract_slots;  // float contraction parts and their dV/dM slots per atom
    int dual_parts, dual_slots;          // the same for the tangent contraction of the loss gradient
    // launchers (stream-ordered, no synchronisation); return the number of kernels launched
    // gather_after (or NULL): an event the force gather waits for (the reverse-pair slots)
    int (*eval_f32)(const EvalCtx<float>&, cudaStream_t, int n_sm, cudaEvent_t* marks, cudaEvent_t gather_after);
    int (*eval_f64)(const EvalCtx<double>&, cudaStream_t, int n_sm, cudaEvent_t* marks, cudaEvent_t gather_after);
    // loss gradient after an evaluation: residuals -> tangent moments -> dual contraction -> dc
    int (*grad_f32)(EvalCtx<float>&, const LossArgs&, cudaStream_t, int n_sm);
    int (*grad_f64)(EvalCtx<double>&, const LossArgs&, cudaStream_t, int n_sm);
};

// Phases timed when profiling is on: marks[k] is recorded before phase k, marks[kPhases] after.
enum { kPhaseMoments = 0, kPhaseContract = 1, kPhasePairgrad = 2, kPhaseGather = 3, kPhases = 4 };

const LevelOps* level_ops(int L);  // nullptr when lev_max is not built

}  // namespace mtp
