// Molecular dynamics with the potential: velocity Verlet, neighbour lists with a skin.
//
// The neighbour list is built once for the search radius R_cut + skin and kept, together with the
// build-time displacements r0_ij and positions x0, while no atom has moved more than skin / 2 (then
// no pair can cross R_cut unseen).  Between rebuilds every step refreshes
//   r_ij = r0_ij + (u_j - u_i),   u = x - x0,
// where u is small, so the float path keeps full float accuracy in r_ij.  Units: Angstrom, fs, eV,
// amu; 1 amu Angstrom^2 / fs^2 = 103.6427 eV.
#include <cuda_runtime.h>
#include "mtp_internal.h"
#include "mtp_common.cuh"

namespace mtp {

namespace {

constexpr double kMvv2eV = 103.642696;  // amu Angstrom^2 fs^-2 in eV

template <class T>
__global__ void k_update_pairs(int n, const int* count, const PairRec<T>* r0, const double* x, const double* x0,
                               PairRec<T>* pr, int* err) {
    const size_t N = (size_t)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double ui0 = x[3 * (size_t)i] - x0[3 * (size_t)i];
        const double ui1 = x[3 * (size_t)i + 1] - x0[3 * (size_t)i + 1];
        const double ui2 = x[3 * (size_t)i + 2] - x0[3 * (size_t)i + 2];
        if (!(isfinite(ui0) && isfinite(ui1) && isfinite(ui2))) atomicOr(err, kErrNonFinite);
        const T fi0 = (T)ui0, fi1 = (T)ui1, fi2 = (T)ui2;
        const int cnt = count[i];
        for (int p = 0; p < cnt; ++p) {
            const size_t o = (size_t)p * N + i;
            PairRec<T> q = r0[o];
            const int j = q.jz & 0xffffff;
            const T uj0 = (T)(x[3 * (size_t)j] - x0[3 * (size_t)j]);
            const T uj1 = (T)(x[3 * (size_t)j + 1] - x0[3 * (size_t)j + 1]);
            const T uj2 = (T)(x[3 * (size_t)j + 2] - x0[3 * (size_t)j + 2]);
            q.x = q.x + (uj0 - fi0);
            q.y = q.y + (uj1 - fi1);
            q.z = q.z + (uj2 - fi2);
            pr[o] = q;
        }
    }
}

__device__ __forceinline__ int species(const int* types, int i, int S) {
    const int z = types[i];  // out-of-range species are reported by the neighbour build
    return z < 0 ? 0 : (z >= S ? S - 1 : z);
}

__global__ void k_kick(int n, int S, double* v, const double* F, const int* types, const double* masses,
                       double half_dt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double s = half_dt / (masses[species(types, i, S)] * kMvv2eV);
        for (int c = 0; c < 3; ++c) v[3 * (size_t)i + c] += s * F[3 * (size_t)i + c];
    }
}

// x += dt v; flags a rebuild when |x - x0| exceeds skin / 2
__global__ void k_drift(int n, double* x, const double* v, const double* x0, double dt, double lim2, int* flag) {
    bool far = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double xn = x[3 * (size_t)i + c] + dt * v[3 * (size_t)i + c];
            x[3 * (size_t)i + c] = xn;
            const double u = xn - x0[3 * (size_t)i + c];
            d2 += u * u;
        }
        far = far || !(d2 <= lim2);  // a NaN displacement forces a rebuild, whose checks report it
    }
    if (__syncthreads_or(far) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_kinetic(int n, int S, const double* v, const int* types, const double* masses, double* out) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v2 = v[3 * (size_t)i] * v[3 * (size_t)i] + v[3 * (size_t)i + 1] * v[3 * (size_t)i + 1] +
                          v[3 * (size_t)i + 2] * v[3 * (size_t)i + 2];
        acc += 0.5 * masses[species(types, i, S)] * kMvv2eV * v2;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, s[0]);
}

int grid_for(int n, int threads, int n_sm) {
    int b = (n + threads - 1) / threads;
    if (b > n_sm * 8) b = n_sm * 8;
    return b < 1 ? 1 : b;
}

}  // namespace

int launch_update_pairs(const NbrState& nb, const double* x, cudaStream_t st, int n_sm) {
    const int n = nb.n_atoms;
    // the evaluation kernels' work queues start at zero (the neighbour build clears them otherwise)
    cudaMemsetAsync(nb.counters.as<int>() + 4, 0, 2 * sizeof(int), st);
    if (nb.fp64)
        k_update_pairs<double><<<grid_for(n, 128, n_sm), 128, 0, st>>>(
            n, nb.count.as<int>(), nb.pr.as<PairRec<double>>(), x, nb.x0.as<double>(), nb.cpr.as<PairRec<double>>(),
            nb.err.as<int>());
    else
        k_update_pairs<float><<<grid_for(n, 128, n_sm), 128, 0, st>>>(
            n, nb.count.as<int>(), nb.pr.as<PairRec<float>>(), x, nb.x0.as<double>(), nb.cpr.as<PairRec<float>>(),
            nb.err.as<int>());
    return 1;
}

int launch_kick(int n, int S, double* v, const double* F, const int* types, const double* masses, double half_dt,
                cudaStream_t st, int n_sm) {
    k_kick<<<grid_for(n, 256, n_sm), 256, 0, st>>>(n, S, v, F, types, masses, half_dt);
    return 1;
}

int launch_drift(int n, double* x, const double* v, const double* x0, double dt, double lim2, int* flag,
                 cudaStream_t st, int n_sm) {
    k_drift<<<grid_for(n, 256, n_sm), 256, 0, st>>>(n, x, v, x0, dt, lim2, flag);
    return 1;
}

int launch_kinetic(int n, int S, const double* v, const int* types, const double* masses, double* out,
                   cudaStream_t st, int n_sm) {
    k_kinetic<<<grid_for(n, 256, n_sm), 256, 0, st>>>(n, S, v, types, masses, out);
    return 1;
}

}  // namespace mtp
