// Shared device structures and helpers of the MTP library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>

namespace mtp {

constexpr int kWarp = 32;
constexpr int kMaxSpecies = 8;  // S*S*N_mu*N_Q coefficients stay within 40 KB of shared memory
constexpr int kMaxRadial = 16;

// device error word bits
enum : int {
    kErrOverflow = 1,   // neighbour list capacity exceeded
    kErrSpecies = 2,    // species index outside [0, S)
    kErrShift = 4,      // |image shift| beyond the packed range
    kErrCellThin = 8,   // cell thinner than the cutoff allows with the supported image range
    kErrTimeout = 16,   // an iteration limit was reached
    kErrSingular = 32,  // singular matrix in the active-set LU
    kErrNonFinite = 64, // a position or cell entry is NaN or infinite
    kErrCell = 128      // a cell with (numerically) zero volume
};

// Inputs and outputs of one evaluation; every array is device memory.
// Three components padded to a 16- (float) or 32-byte (double) vector: one load or store per pair.
template <class T>
struct alignas(4 * sizeof(T)) Vec4 {
    T x, y, z, w;
};

// One neighbour pair of the slot-major lists: r_ij and (neighbour index | species << 24), written
// and read as one record (16 bytes in float, two 16-byte halves in double).
template <class T>
struct PairRec;
template <>
struct __align__(16) PairRec<float> {
    float x, y, z;
    int jz;
};
template <>
struct __align__(32) PairRec<double> {
    double x, y, z;
    int jz, pad;
};

template <class T>
struct EvalCtx {
    int n_atoms;      // atoms in the batch
    int n_cfg;        // configurations in the batch
    int cap;          // neighbour slots per atom (slot-major arrays have stride n_atoms)
    int S, NQ;        // species, radial basis size
    T rmin, rcut, inv_span;
    const int* types;     // [n]
    const int* cfg_of;    // [n] atom -> configuration
    const int* cfg_off;   // [n_cfg + 1] first atom of each configuration
    const int* count;     // [n] neighbours of each atom
    const PairRec<T>* pr;  // [cap][n] r_ij and neighbour index | species << 24
    const int* rev;       // [cap][n] slot of the reverse pair in the neighbour's list, -1 if absent
    const T* c;           // [S][S][NMU][NQ] radial coefficients
    const T* xi;          // [M]
    const T* seed;        // [V] adjoint seed: xi at the value index of each basis function
    const int* basis_value;  // [M]
    const unsigned long long* fwd_ops;  // forward program rows (32 packed ops per row)
    const int* fwd_layer_end;
    int fwd_layers;
    const unsigned long long* adj_ops;  // adjoint program rows
    const int* adj_layer_end;
    int adj_layers;
    const float* weights;               // [n_weights] op weights
    int n_weights;
    int* queue;           // [2] work-queue counters of k_moments and k_pairgrad (zero at the start of an evaluation)
    int tpa;              // threads per atom in the pair-gradient, gather and loss-gradient kernels (1, 2, 4 or 8)
    int tpa_m;            // threads per atom in the moments kernel
    T* mom;               // [ceil(n/32)][C][32] moment components (tile layout)
    T* adjm;              // [ceil(n/32)][C][32] dV/dM
    T* aslots;            // [ceil(n/32)][NSLOT][32] dV/dM shares of the contraction parts (float path)
    T* epart;             // [NPART][n] site-energy shares of the contraction parts (float path)
    Vec4<T>* g;           // [cap][n] dV_i/dr_ij (x, y, z, unused): one vector load per pair
    double* energy;       // [n_cfg] (accumulated; zeroed by the caller) or NULL
    double* site;         // [n] or NULL
    double* b_atoms;      // [n][M] or NULL
    double* b_rows;       // [n_cfg][M] (accumulated) or NULL
    double* forces;       // [n][3] or NULL
    double* virial;       // [n_cfg][9] (accumulated) or NULL
    int* err;
    // training-loss gradient (Sec. 2.2): residual directions and outputs
    const T* gD;          // [n][3] D_i = 2 s_f w_f (F_i - F_i^ref)
    const T* geps;        // [n_cfg][9] eps_k = 2 s_s w_s (W_k - W_k^ref)
    const double* gew;    // [n_cfg] e_k = 2 s_e w_e (E_k - E_k^ref)
    T* momt;              // tangent of the moments along u (tile layout)
    T* adjmt;             // tangent of dV/dM (tile layout)
    double* dxi;          // [M] accumulated dL/dxi
    T* dslots;            // [2][ceil(n/32)][NDSLOT][32] dV/dM and its tangent, per tangent-contraction part
    double* dxt;          // [ceil(n/32)][M] per-tile shares of dL/dxi from the tangent contraction
    double* dc;           // [S][S][NMU][NQ] accumulated dL/dc
    double* dc_rows;      // [n_cfg][S][S][NMU][NQ] per-configuration dE_k/dc (Jacobian rows) or NULL
};

// Loss (Sec. 2.2): residuals and the directions of the gradient.  Scalings of Eqs. 7, 11, 12.
struct LossArgs {
    int n_atoms, n_cfg, scaling;  // 0 molecules, 1 structures, 2 vibrations
    double we, wf, ws;
    const int* cfg_off;
    const int* cfg_of;
    const double* energy;   // [K] model
    const double* forces;   // [N][3] model
    const double* virial;   // [K][9] model
    const double* e_ref;
    const double* f_ref;
    const double* w_ref;
    double* loss;           // [1] accumulated
    double* gew;            // [K]
    int loss_only;          // 1: residuals and loss only, no gradient kernels
    int jacobian;           // 1: per-configuration dE/dc (the caller set e_k = 1, D = 0, eps = 0)
};

__host__ __device__ inline void loss_scales(int kind, double n, double* se, double* sf, double* ss) {
    if (kind == 0) {
        *se = 1.0; *sf = 1.0; *ss = 1.0;
    } else if (kind == 1) {
        *se = 1.0 / (n * n); *sf = 1.0 / n; *ss = 1.0 / (n * n);
    } else {
        *se = 1.0 / n; *sf = 1.0; *ss = 1.0 / n;
    }
}

// A timing event on a stream; inside a stream capture it becomes an externally visible record node
// (a plain record there is only a dependency and cannot be timed).
inline void record_mark(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

// Programmatic dependent launch (sm_90 and later).  A kernel started by launch_pdl may begin while
// the previous kernel of its stream is still running; before its first global-memory access it
// calls pdl_wait, which returns once that kernel has completed and its writes are visible (a no-op
// for a kernel launched the ordinary way).  pdl_trigger lets the next kernel of the stream start
// launching; it changes no ordering of memory accesses.  Kernels of the evaluation chain call both
// at entry, so only the launch latency of the next kernel overlaps the current one.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

template <class... P, class... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t st,
                              A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mtp
