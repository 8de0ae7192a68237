// Batched structure relaxation (the paper's relaxation of candidate structures, Sec. 5: energy
// minimisation over atomic positions and lattice vectors, ending relaxed or at the first
// extrapolative configuration).  The minimiser is FIRE (Bitzek et al., Phys. Rev. Lett. 97, 170201,
// 2006), which the paper does not name: semi-implicit Euler steps with unit masses, the velocity
// mixed towards the force, step growth after N_min = 5 downhill steps (f_inc 1.1, f_a 0.99) and a
// reset when the power F.v is not positive (f_dec 0.5, a_start 0.1).  The cell moves through the
// deformation gradient D of the starting cell: H = H0 D^T, x = u D^T; the force on u is F D and
// the force on D is W D^-T / N (W the virial).  Every configuration of the batch keeps its own
// state; one block per configuration updates it after each batched evaluation.
#include <cuda_runtime.h>
#include "mtp_common.cuh"
#include "mtp_internal.h"

namespace mtp {

namespace {

constexpr int kRelaxThreads = 256;
constexpr int kNmin = 5;
constexpr double kFinc = 1.1, kFdec = 0.5, kAstart = 0.1, kFa = 0.99;

__device__ __forceinline__ int cfg_of_atom(const int* off, int K, int i) {
    int lo = 0, hi = K;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// x = u D^T per atom and H = H0 D^T per configuration
__global__ void k_relax_map(int n, int K, const int* off, const double* u, const double* D, const double* H0,
                            double* x, double* H) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const double* d = D + 9 * (size_t)cfg_of_atom(off, K, t);
        for (int a = 0; a < 3; ++a)
            x[3 * (size_t)t + a] = u[3 * (size_t)t] * d[3 * a] + u[3 * (size_t)t + 1] * d[3 * a + 1] +
                                   u[3 * (size_t)t + 2] * d[3 * a + 2];
    } else if (t < n + K) {
        const int k = t - n;
        const double* d = D + 9 * (size_t)k;
        const double* h = H0 + 9 * (size_t)k;
        for (int r = 0; r < 3; ++r)
            for (int a = 0; a < 3; ++a)
                H[9 * (size_t)k + 3 * r + a] = h[3 * r] * d[3 * a] + h[3 * r + 1] * d[3 * a + 1] + h[3 * r + 2] * d[3 * a + 2];
    }
}

__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// One FIRE iteration of every running configuration (block k = configuration k), in the order of
// the minimiser: finite forces, extrapolation stop, convergence, step limit, then the update.
__global__ void __launch_bounds__(kRelaxThreads) k_fire(RelaxArgs a, int step) {
    __shared__ double sh[kRelaxThreads];
    __shared__ double sD[9], sDi[9], sfD[9], sv[9];
    const int k = blockIdx.x;
    if (a.status[k] != 0) return;  // finished: frozen
    const int i0 = a.off[k], i1 = a.off[k + 1], nk = i1 - i0;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < 9; ++q) sD[q] = a.D[9 * (size_t)k + q];
        // D^-1 (3 x 3) by cofactors
        const double* d = sD;
        const double det = d[0] * (d[4] * d[8] - d[5] * d[7]) - d[1] * (d[3] * d[8] - d[5] * d[6]) +
                           d[2] * (d[3] * d[7] - d[4] * d[6]);
        const double id = 1.0 / det;
        sDi[0] = (d[4] * d[8] - d[5] * d[7]) * id; sDi[1] = (d[2] * d[7] - d[1] * d[8]) * id;
        sDi[2] = (d[1] * d[5] - d[2] * d[4]) * id; sDi[3] = (d[5] * d[6] - d[3] * d[8]) * id;
        sDi[4] = (d[0] * d[8] - d[2] * d[6]) * id; sDi[5] = (d[2] * d[3] - d[0] * d[5]) * id;
        sDi[6] = (d[3] * d[7] - d[4] * d[6]) * id; sDi[7] = (d[1] * d[6] - d[0] * d[7]) * id;
        sDi[8] = (d[0] * d[4] - d[1] * d[3]) * id;
        // force on D: W D^-T / N  (fD[r][c] = sum_s W[r][s] Di[c][s] / N)
        const double* W = a.W + 9 * (size_t)k;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                sfD[3 * r + c] = a.relax_cell
                                     ? (W[3 * r] * sDi[3 * c] + W[3 * r + 1] * sDi[3 * c + 1] + W[3 * r + 2] * sDi[3 * c + 2]) /
                                           (double)(nk > 0 ? nk : 1)
                                     : 0.0;
        for (int q = 0; q < 9; ++q) sv[q] = a.vD[9 * (size_t)k + q];
    }
    __syncthreads();
    // reductions over the configuration's coordinates: force on u_i is F_i D
    double P = 0.0, ff = 0.0, vv = 0.0, fmaxv = 0.0;
    bool finite = true;
    for (int i = i0 + tid; i < i1; i += blockDim.x) {
        const double* F = a.F + 3 * (size_t)i;
        const double* v = a.vu + 3 * (size_t)i;
        const double* u = a.u + 3 * (size_t)i;
        for (int c = 0; c < 3; ++c) {
            const double f = F[0] * sD[c] + F[1] * sD[3 + c] + F[2] * sD[6 + c];
            P += f * v[c];
            ff += f * f;
            vv += v[c] * v[c];
            fmaxv = fmax(fmaxv, fabs(F[c]));
            finite = finite && isfinite(f) && isfinite(u[c]) && isfinite(F[c]);
        }
    }
    if (tid < 9 && a.relax_cell) {
        P += sfD[tid] * sv[tid];
        ff += sfD[tid] * sfD[tid];
        vv += sv[tid] * sv[tid];
        finite = finite && isfinite(sfD[tid]) && isfinite(sD[tid]);
    }
    P = block_sum(P, sh);
    ff = block_sum(ff, sh);
    vv = block_sum(vv, sh);
    fmaxv = block_max(fmaxv, sh);
    const bool all_finite = __syncthreads_and(finite);
    // convergence: max |F| <= fmax and max |W| / volume <= smax (the cell only when it relaxes)
    bool conv = fmaxv <= a.fmax;
    if (a.relax_cell) {
        const double* W = a.W + 9 * (size_t)k;
        const double* H = a.H + 9 * (size_t)k;
        const double vol = fabs(H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                                H[2] * (H[3] * H[7] - H[4] * H[6]));
        double wm = 0.0;
        for (int q = 0; q < 9; ++q) wm = fmax(wm, fabs(W[q]));
        conv = conv && wm / vol <= a.smax;
    }
    const bool stop = a.gamma && a.gamma[k] >= a.gamma_break;
    int st = 0;
    if (!all_finite)
        st = kRelaxDiverged;
    else if (stop)
        st = kRelaxStopped;
    else if (conv)
        st = kRelaxConverged;
    else if (step == a.max_steps)
        st = kRelaxStepLimit;
    if (st) {
        if (tid == 0) {
            a.status[k] = st;
            a.steps[k] = step;
            a.e_final[k] = a.E[k];
        }
        return;
    }
    // FIRE update (uniform over the block)
    double dt = a.dt[k], alpha = a.alpha[k];
    int npos = a.npos[k];
    double mix_v = 1.0, mix_f = 0.0;
    bool zero_v = false;
    if (P > 0.0) {
        mix_v = 1.0 - alpha;
        mix_f = ff > 0.0 ? alpha * sqrt(vv) / sqrt(ff) : 0.0;
        ++npos;
        if (npos > kNmin) {
            dt = fmin(dt * kFinc, a.dt_max);
            alpha *= kFa;
        }
    } else {
        zero_v = true;
        dt *= kFdec;
        alpha = kAstart;
        npos = 0;
    }
    for (int i = i0 + tid; i < i1; i += blockDim.x) {
        const double* F = a.F + 3 * (size_t)i;
        double* v = a.vu + 3 * (size_t)i;
        double* u = a.u + 3 * (size_t)i;
        for (int c = 0; c < 3; ++c) {
            const double f = F[0] * sD[c] + F[1] * sD[3 + c] + F[2] * sD[6 + c];
            double vn = zero_v ? 0.0 : mix_v * v[c] + mix_f * f;
            vn = vn + dt * f;
            v[c] = vn;
            u[c] = u[c] + dt * vn;
        }
    }
    if (tid < 9 && a.relax_cell) {
        double vn = zero_v ? 0.0 : mix_v * sv[tid] + mix_f * sfD[tid];
        vn = vn + dt * sfD[tid];
        a.vD[9 * (size_t)k + tid] = vn;
        a.D[9 * (size_t)k + tid] = sD[tid] + dt * vn;
    }
    if (tid == 0) {
        a.dt[k] = dt;
        a.alpha[k] = alpha;
        a.npos[k] = npos;
    }
}

// initial state: u = x, D = I, velocities 0, dt, alpha = a_start, npos = 0, status 0 (running)
__global__ void k_relax_init(int n, int K, const double* x, double* u, double* vu, double* D, double* vD, double* dt,
                             double* alpha, int* npos, int* status, int* steps, const int* off, double dt0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 3 * n) {
        u[t] = x[t];
        vu[t] = 0.0;
    }
    if (t < K) {
        for (int q = 0; q < 9; ++q) {
            D[9 * (size_t)t + q] = (q % 4 == 0) ? 1.0 : 0.0;
            vD[9 * (size_t)t + q] = 0.0;
        }
        dt[t] = dt0;
        alpha[t] = kAstart;
        npos[t] = 0;
        steps[t] = 0;
        status[t] = off[t + 1] > off[t] ? 0 : kRelaxConverged;  // an empty configuration has nothing to do
    }
}

}  // namespace

int launch_relax_init(const RelaxArgs& a, int n, int K, const double* x, double dt0, cudaStream_t st) {
    const int t = 3 * n > K ? 3 * n : K;
    k_relax_init<<<(t + 255) / 256, 256, 0, st>>>(n, K, x, a.u, a.vu, a.D, a.vD, a.dt, a.alpha, a.npos, a.status,
                                                  a.steps, a.off, dt0);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_relax_map(int n, int K, const int* off, const double* u, const double* D, const double* H0, double* x,
                     double* H, cudaStream_t st) {
    k_relax_map<<<(n + K + 255) / 256, 256, 0, st>>>(n, K, off, u, D, H0, x, H);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_fire(const RelaxArgs& a, int K, int step, cudaStream_t st) {
    k_fire<<<K, kRelaxThreads, 0, st>>>(a, step);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mtp
