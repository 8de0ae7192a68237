// Training optimiser on the device (Sec. 2.2: theta = (xi, c) minimises the loss of Eqs. 7, 11, 12;
// the paper names no algorithm): limited-memory BFGS (Nocedal and Wright, Algorithms 7.4 and 7.5)
// with a backtracking line search on the Armijo condition.  The parameter vector, the gradient, the
// search direction and the (s, y) history stay in device memory; every kernel here is one block
// (theta has at most a few thousand entries) with fixed-order reductions, so the iteration is
// deterministic given the gradients.
#include <cuda_runtime.h>
#include "mtp_common.cuh"
#include "mtp_internal.h"

namespace mtp {

namespace {

constexpr int kTrainThreads = 1024;

__device__ double block_sum_train(double v, double* sh) {
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

__device__ double block_max_train(double v, double* sh) {
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

// d = -H g by the two-loop recursion over the pairs held in ring slots order[0..k-1] (oldest first)
// of S, Y [history][P]; scalars out: [0] g.d, [1] max |g|.
__global__ void __launch_bounds__(kTrainThreads) k_lbfgs_direction(int P, int k, const int* order, const double* S,
                                                                   const double* Y, const double* g, double* d,
                                                                   double* alpha, double* scalars) {
    __shared__ double sh[kTrainThreads];
    for (int e = threadIdx.x; e < P; e += blockDim.x) d[e] = g[e];
    __syncthreads();
    for (int q = k - 1; q >= 0; --q) {  // newest to oldest
        const double* s = S + (size_t)order[q] * P;
        const double* y = Y + (size_t)order[q] * P;
        double sq = 0.0, ys = 0.0;
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            sq += s[e] * d[e];
            ys += y[e] * s[e];
        }
        sq = block_sum_train(sq, sh);
        ys = block_sum_train(ys, sh);
        const double a = sq / ys;
        if (threadIdx.x == 0) alpha[q] = a;
        for (int e = threadIdx.x; e < P; e += blockDim.x) d[e] -= a * y[e];
        __syncthreads();
    }
    double scale;
    if (k > 0) {
        const double* s = S + (size_t)order[k - 1] * P;
        const double* y = Y + (size_t)order[k - 1] * P;
        double sy = 0.0, yy = 0.0;
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            sy += s[e] * y[e];
            yy += y[e] * y[e];
        }
        sy = block_sum_train(sy, sh);
        yy = block_sum_train(yy, sh);
        scale = sy / yy;
    } else {
        double gm = 0.0;
        for (int e = threadIdx.x; e < P; e += blockDim.x) gm = fmax(gm, fabs(g[e]));
        gm = block_max_train(gm, sh);
        scale = 1.0 / fmax(1.0, gm);
    }
    for (int e = threadIdx.x; e < P; e += blockDim.x) d[e] *= scale;
    __syncthreads();
    for (int q = 0; q < k; ++q) {  // oldest to newest
        const double* s = S + (size_t)order[q] * P;
        const double* y = Y + (size_t)order[q] * P;
        double yq = 0.0, ys = 0.0;
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            yq += y[e] * d[e];
            ys += y[e] * s[e];
        }
        yq = block_sum_train(yq, sh);
        ys = block_sum_train(ys, sh);
        const double b = yq / ys;
        const double a = alpha[q];
        for (int e = threadIdx.x; e < P; e += blockDim.x) d[e] += s[e] * (a - b);
        __syncthreads();
    }
    double gd = 0.0, gm = 0.0;
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        d[e] = -d[e];
        gd += g[e] * d[e];
        gm = fmax(gm, fabs(g[e]));
    }
    gd = block_sum_train(gd, sh);
    gm = block_max_train(gm, sh);
    if (threadIdx.x == 0) {
        scalars[0] = gd;
        scalars[1] = gm;
    }
}

// theta_trial = theta + t d, and the model's parameter arrays (xi, c and the adjoint seed of xi at
// the value slot of each basis function) in the model's precision
template <class T>
__global__ void __launch_bounds__(kTrainThreads) k_train_set(int P, int m, const double* theta, const double* d,
                                                             double t, double* trial, T* xi, T* c, T* seed, int V,
                                                             const int* basis_value) {
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        const double v = theta[e] + t * d[e];
        trial[e] = v;
        if (e < m)
            xi[e] = (T)v;
        else
            c[e - m] = (T)v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the seed in a fixed order (several basis functions may share a slot)
        for (int v = 0; v < V; ++v) seed[v] = T(0);
        for (int a = 0; a < m; ++a) seed[basis_value[a]] += (T)trial[a];
    }
}

// s = trial - theta, y = g_new - g into ring slot `slot`; scalars out: [2] s.y, [3] |s|, [4] |y|,
// [5] max |g_new|
__global__ void __launch_bounds__(kTrainThreads) k_lbfgs_pair(int P, const double* theta, const double* trial,
                                                              const double* g, const double* g_new, double* S,
                                                              double* Y, int slot, double* scalars) {
    __shared__ double sh[kTrainThreads];
    double sy = 0.0, ss = 0.0, yy = 0.0, gm = 0.0;
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        const double s = trial[e] - theta[e], y = g_new[e] - g[e];
        S[(size_t)slot * P + e] = s;
        Y[(size_t)slot * P + e] = y;
        sy += s * y;
        ss += s * s;
        yy += y * y;
        gm = fmax(gm, fabs(g_new[e]));
    }
    sy = block_sum_train(sy, sh);
    ss = block_sum_train(ss, sh);
    yy = block_sum_train(yy, sh);
    gm = block_max_train(gm, sh);
    if (threadIdx.x == 0) {
        scalars[2] = sy;
        scalars[3] = sqrt(ss);
        scalars[4] = sqrt(yy);
        scalars[5] = gm;
    }
}

}  // namespace

int launch_lbfgs_direction(int P, int k, const int* order, const double* S, const double* Y, const double* g,
                           double* d, double* alpha, double* scalars, cudaStream_t st) {
    k_lbfgs_direction<<<1, kTrainThreads, 0, st>>>(P, k, order, S, Y, g, d, alpha, scalars);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <class T>
int launch_train_set(int P, int m, const double* theta, const double* d, double t, double* trial, T* xi, T* c, T* seed,
                     int V, const int* basis_value, cudaStream_t st) {
    k_train_set<T><<<1, kTrainThreads, 0, st>>>(P, m, theta, d, t, trial, xi, c, seed, V, basis_value);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}
template int launch_train_set<float>(int, int, const double*, const double*, double, double*, float*, float*, float*,
                                     int, const int*, cudaStream_t);
template int launch_train_set<double>(int, int, const double*, const double*, double, double*, double*, double*,
                                      double*, int, const int*, cudaStream_t);

int launch_lbfgs_pair(int P, const double* theta, const double* trial, const double* g, const double* g_new,
                      double* S, double* Y, int slot, double* scalars, cudaStream_t st) {
    k_lbfgs_pair<<<1, kTrainThreads, 0, st>>>(P, theta, trial, g, g_new, S, Y, slot, scalars);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mtp
