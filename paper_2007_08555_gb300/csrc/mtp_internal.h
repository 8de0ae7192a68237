// Host-side internals of the MTP library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include "mtp_level.h"

namespace mtp {

// A device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t want) {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t b = want + want / 4 + 256;
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

struct CellDesc {
    double H[9];
    float Hi[9];  // inverse cell (float: it only places atoms in bins and lattice wraps)
    float hn[9];  // lattice vectors divided by the bin counts, rows
    float hhi[9], hlo[9];  // lattice vectors as float pairs (hi + lo = H to ~2^-48)
    float inv_n[3];
    int n[3], c[3];
    int bin0, nbins;
};

// Neighbour list in slot-major layout (stride = number of atoms).
struct NbrState {
    int n_atoms = 0, n_cfg = 0, cap = 0;
    bool fp64 = false;
    double rsearch = 0.0;
    DevBuf count, pr, rev, keys_am;  // pr: [cap][n] PairRec (r_ij, neighbour | species << 24)
    DevBuf cfg_of, desc, atom_bin, atom_wrap, atom_local, atom_wp, bin_count, bin_start, atom_slot, bin_atoms, counters;
    DevBuf err;
    // reuse with a skin: positions at the build and the pair records with r_ij refreshed for the
    // current positions
    DevBuf x0, cpr;
    bool has_x0 = false;
};

// Build the neighbour list of a batch (device inputs).  r_ij are written in float or double.
// With a side stream, the reverse-pair slots (needed only by the force gather) are computed there,
// after `fork` is recorded on st, and `join` is recorded when they are done: the caller makes the
// gather wait on `join`.  Returns the number of kernels launched, or -1 on a CUDA error
// (cudaGetLastError holds it).
int build_neighbors(NbrState& nb, int n_cfg, int n_atoms, const int* cfg_off, const double* pos,
                    const int* types, const double* cells, double rsearch, bool fp64, int cap,
                    cudaStream_t st, int n_species, cudaStream_t side = nullptr, cudaEvent_t fork = nullptr,
                    cudaEvent_t join = nullptr);

// Exclusive prefix sum of n ints: out[0..n] with out[n] = total; tmp holds >= scan_tmp_ints(n) ints.
size_t scan_tmp_ints(int n);
int scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t st);

// Active set (mtp_maxvol.cu)
int launch_maxvol(int n, int m, const double* B, double* Bs, double* D, double* W, int* perm, int* sel, double* A,
                  double* Ai, double* C, double tol, int max_iter, int* status, int* swaps, double* gmax,
                  cudaStream_t st, int start_given = 0);
int launch_invert(int m, const double* A, double* Ai, double* W, int* status, cudaStream_t st);
template <class T>
int launch_grade(int n, int m, const T* B, int ldb, const T* Ai, unsigned long long* gbits, cudaStream_t st);
// out[r][q] = in[r][cols[q]] (rows x w_out from rows x w_in)
int launch_gather_columns(int rows, int w_in, const double* in, int w_out, const int* cols, double* out,
                          cudaStream_t st);

// Tensor-core grade (mtp_grade_tc.cu): digits of (A D)^-1 prepared once per active set (m <= 480),
// then gamma of n rows (gbits cleared by the launcher); return launches or -1.
size_t grade_tc_digit_bytes(int m);
int launch_grade_tc_prep(int m, const double* A, const double* Ai, void* digits, int* ecol, float* cscale,
                         cudaStream_t st);
int launch_grade_tc(int n, int m, const double* B, int ldb, const void* digits, const int* ecol, const float* cscale,
                    unsigned long long* gbits, int* err, cudaStream_t st, int n_sm);

// Batched relaxation (mtp_relax.cu): FIRE state of every configuration and the evaluation at the
// current coordinates (forces, virial, energy, cell, grade or NULL).
enum { kRelaxRunning = 0, kRelaxConverged = 1, kRelaxStopped = 2, kRelaxStepLimit = 3, kRelaxDiverged = 4 };
struct RelaxArgs {
    const int* off;
    int relax_cell, max_steps;
    double fmax, smax, gamma_break, dt_max;
    const double* F;      // [n][3]
    const double* W;      // [K][9]
    const double* E;      // [K]
    const double* H;      // [K][9] current cells
    const double* gamma;  // [K] or NULL
    double *u, *vu, *D, *vD, *dt, *alpha, *e_final;
    int *npos, *status, *steps;
};
int launch_relax_init(const RelaxArgs& a, int n, int K, const double* x, double dt0, cudaStream_t st);
int launch_relax_map(int n, int K, const int* off, const double* u, const double* D, const double* H0, double* x,
                     double* H, cudaStream_t st);
int launch_fire(const RelaxArgs& a, int K, int step, cudaStream_t st);

// Training optimiser (mtp_train.cu): L-BFGS direction, parameter update, history pair.
int launch_lbfgs_direction(int P, int k, const int* order, const double* S, const double* Y, const double* g,
                           double* d, double* alpha, double* scalars, cudaStream_t st);
template <class T>
int launch_train_set(int P, int m, const double* theta, const double* d, double t, double* trial, T* xi, T* c, T* seed,
                     int V, const int* basis_value, cudaStream_t st);
int launch_lbfgs_pair(int P, const double* theta, const double* trial, const double* g, const double* g_new,
                      double* S, double* Y, int slot, double* scalars, cudaStream_t st);

// Molecular dynamics helpers (mtp_md.cu).  The refreshed r_ij go to nb.cx/cy/cz.
int launch_update_pairs(const NbrState& nb, const double* x, cudaStream_t st, int n_sm);
int launch_kick(int n, int S, double* v, const double* F, const int* types, const double* masses, double half_dt,
                cudaStream_t st, int n_sm);
int launch_drift(int n, double* x, const double* v, const double* x0, double dt, double lim2, int* flag,
                 cudaStream_t st, int n_sm);
int launch_kinetic(int n, int S, const double* v, const int* types, const double* masses, double* out,
                   cudaStream_t st, int n_sm);

// CSR export of the neighbour list with exact double-precision r_ij.
int export_neighbors(const NbrState& nb, const double* pos, const int* offsets, int* nbr_j, int* nbr_s,
                     double* r_ij, cudaStream_t st);

}  // namespace mtp
