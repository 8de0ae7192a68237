// Active set and extrapolation grade of Sec. 2.3 (D-optimality, MaxVol of Goreinov et al. 2010).
//
// k_maxvol (one CTA, double precision, all loops bounded):
//   0. columns are scaled by 1 / max |column| (the grades and the selection are invariant under
//      B -> B D, and the scaled matrix is far better conditioned);
//   1. start rows: the pivot rows of Gaussian elimination with partial pivoting on the tall
//      matrix B (n_rows x m); ties go to the smaller current row position (or, for the select-add
//      update, the first m rows: the current active set stacked above the candidates);
//   2. A^-1 of A = B[sel] by Gauss-Jordan elimination with partial pivoting;
//   3. C = B A^-1 for every row;
//   4. repeat at most max_iter times: (k, j) = argmax |C_kj| (ties: smallest k, then smallest j);
//      stop when |C_kj| <= 1 + tol (tol = 1e-3); otherwise row k replaces active row j, and A^-1 and C follow
//      by the rank-one (Sherman-Morrison) update  C <- C - C[:,j] (C[k,:] - e_j) / C_kj.
//   A^-1 is recomputed from scratch at the end.
// k_grade: gamma_r = max_j |(b_r A^-1)_j| for many rows; 64x64 output tiles through shared memory,
//   the row maxima are combined with an atomic max on the bit pattern (gamma >= 0); a NaN in a row
//   of b A^-1 gives gamma = +inf, so a broken configuration reads as extrapolating.
#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <mutex>
#include "../../include/mtp.h"
#include "mtp_common.cuh"

namespace mtp {

namespace {

constexpr int kMvThreads = 1024;

struct ArgMax {
    double v;
    int idx;
};

// block-wide argmax of |value| (ties -> smallest index); every thread returns the winner
__device__ ArgMax block_argmax(double v, int idx, ArgMax* sbuf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 < idx)) {
            v = v2;
            idx = i2;
        }
    }
    if (lane == 0) sbuf[warp] = {v, idx};
    __syncthreads();
    if (warp == 0) {
        ArgMax a = lane < (int)(blockDim.x >> 5) ? sbuf[lane] : ArgMax{-1.0, 0x7fffffff};
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, a.v, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, a.idx, o);
            if (v2 > a.v || (v2 == a.v && i2 < a.idx)) {
                a.v = v2;
                a.idx = i2;
            }
        }
        if (lane == 0) sbuf[32] = a;
    }
    __syncthreads();
    const ArgMax r = sbuf[32];
    __syncthreads();
    return r;
}

// inverse of the m x m matrix A (row-major) into Ai, Gauss-Jordan with partial pivoting on a
// work copy W [m][2m].  Returns false if a pivot is exactly zero.
__device__ bool gauss_jordan(const double* A, double* Ai, double* W, int m, ArgMax* sbuf, int* s_flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = 2 * m;
    for (int e = tid; e < m * w; e += nt) {
        const int r = e / w, c = e % w;
        W[e] = c < m ? A[r * m + c] : (c - m == r ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int r = k + tid; r < m; r += nt) {
            const double v = fabs(W[r * w + k]);
            if (v > best || (v == best && r < bi)) {
                best = v;
                bi = r;
            }
        }
        const ArgMax p = block_argmax(best, bi, sbuf);
        if (p.v == 0.0) return false;
        if (p.idx != k)
            for (int c = tid; c < w; c += nt) {
                const double t = W[k * w + c];
                W[k * w + c] = W[p.idx * w + c];
                W[p.idx * w + c] = t;
            }
        __syncthreads();
        const double inv = 1.0 / W[k * w + k];
        __syncthreads();  // every thread has read the pivot before row k is scaled
        for (int c = tid; c < w; c += nt) W[k * w + c] *= inv;
        __syncthreads();
        for (int e = tid; e < m * w; e += nt) {
            const int r = e / w, c = e % w;
            if (r != k) {
                const double f = W[r * w + k];
                if (c != k) W[e] -= f * W[k * w + c];
            }
        }
        __syncthreads();
        for (int r = tid; r < m; r += nt)
            if (r != k) W[r * w + k] = 0.0;
        __syncthreads();
    }
    for (int e = tid; e < m * m; e += nt) Ai[e] = W[(e / m) * w + m + (e % m)];
    __syncthreads();
    (void)s_flag;
    return true;
}

__global__ void __launch_bounds__(kMvThreads) k_maxvol(int n, int m, const double* Braw, double* Bs, double* D,
                                                       double* W, int* perm, int* sel, double* A, double* Ai, double* C,
                                                       double tol, int max_iter, int* status, int* swaps_out,
                                                       double* gmax_out, int start_given) {
    __shared__ ArgMax sbuf[33];
    __shared__ int s_flag;
    const int tid = threadIdx.x, nt = blockDim.x;
    // 0. column equilibration: gamma and the selection do not change under B -> B D
    for (int c = tid; c < m; c += nt) {
        double mx = 0.0;
        for (int r = 0; r < n; ++r) mx = fmax(mx, fabs(Braw[(size_t)r * m + c]));
        D[c] = mx > 0.0 ? 1.0 / mx : 0.0;
    }
    __syncthreads();
    for (int c = 0; c < m; ++c)
        if (D[c] == 0.0) {
            if (tid == 0) *status = kErrSingular;
            return;
        }
    for (int e = tid; e < n * m; e += nt) Bs[e] = Braw[e] * D[e % m];
    __syncthreads();
    const double* B = Bs;
    if (start_given) {  // select-add: start from the first m rows (the current active set)
        for (int j = tid; j < m; j += nt) sel[j] = j;
        __syncthreads();
        goto have_start;
    }
    // 1. pivot rows of LU with partial pivoting (row interchanges tracked in perm)
    for (int e = tid; e < n * m; e += nt) W[e] = B[e];
    for (int r = tid; r < n; r += nt) perm[r] = r;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int r = k + tid; r < n; r += nt) {
            const double v = fabs(W[perm[r] * m + k]);
            if (v > best || (v == best && r < bi)) {
                best = v;
                bi = r;
            }
        }
        const ArgMax p = block_argmax(best, bi, sbuf);
        if (p.v == 0.0) {
            if (tid == 0) *status = kErrSingular;
            return;
        }
        if (tid == 0 && p.idx != k) {
            const int t = perm[k];
            perm[k] = perm[p.idx];
            perm[p.idx] = t;
        }
        __syncthreads();
        const int pk = perm[k];
        const double piv = W[pk * m + k];
        const int rows = n - k - 1, cols = m - k - 1;
        for (int e = tid; e < rows * (cols + 1); e += nt) {
            const int rr = k + 1 + e / (cols + 1), c = k + e % (cols + 1);
            const int pr = perm[rr];
            const double l = W[pr * m + k] / piv;
            if (c > k) W[pr * m + c] -= l * W[pk * m + c];
        }
        __syncthreads();
        // the multipliers are no longer needed in column k (kept implicit)
    }
    for (int j = tid; j < m; j += nt) sel[j] = perm[j];
    __syncthreads();
have_start:
    // 2. A and its inverse
    for (int e = tid; e < m * m; e += nt) A[e] = B[sel[e / m] * m + (e % m)];
    __syncthreads();
    if (!gauss_jordan(A, Ai, W, m, sbuf, &s_flag)) {
        if (tid == 0) *status = kErrSingular;
        return;
    }
    // 3. C = B A^-1
    for (int e = tid; e < n * m; e += nt) {
        const int r = e / m, c = e % m;
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += B[r * m + k] * Ai[k * m + c];
        C[e] = s;
    }
    __syncthreads();
    // 4. swaps
    int swaps = 0;
    double g = 0.0;
    for (int it = 0; it <= max_iter; ++it) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int e = tid; e < n * m; e += nt) {
            const double v = fabs(C[e]);
            if (v > best || (v == best && e < bi)) {
                best = v;
                bi = e;
            }
        }
        const ArgMax p = block_argmax(best, bi, sbuf);
        g = p.v;
        if (p.v <= 1.0 + tol) break;
        if (it == max_iter) {
            if (tid == 0) *status = kErrTimeout;
            break;
        }
        const int k = p.idx / m, j = p.idx % m;
        const double ckj = C[p.idx];
        // Ai <- Ai - Ai[:,j] (C[k,:] - e_j) / ckj ; C <- C - C[:,j] (C[k,:] - e_j) / ckj
        // (read the column and the row before writing: stage them in W)
        for (int t = tid; t < m; t += nt) {
            W[t] = C[k * m + t] - (t == j ? 1.0 : 0.0);  // row
            W[m + t] = Ai[t * m + j];                     // column of Ai
        }
        for (int r = tid; r < n; r += nt) W[2 * m + r] = C[r * m + j];
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) Ai[e] -= W[m + e / m] * W[e % m] / ckj;
        for (int e = tid; e < n * m; e += nt) C[e] -= W[2 * m + e / m] * W[e % m] / ckj;
        if (tid == 0) sel[j] = k;
        __syncthreads();
        ++swaps;
    }
    // final A (unscaled rows of B) and A^-1 = D (A D)^-1, the inverse recomputed from scratch
    for (int e = tid; e < m * m; e += nt) A[e] = B[sel[e / m] * m + (e % m)];
    __syncthreads();
    if (!gauss_jordan(A, Ai, W, m, sbuf, &s_flag)) {
        if (tid == 0) *status = kErrSingular;
        return;
    }
    for (int e = tid; e < m * m; e += nt) {
        Ai[e] *= D[e / m];
        A[e] = Braw[(size_t)sel[e / m] * m + (e % m)];
    }
    __syncthreads();
    if (tid == 0) {
        *swaps_out = swaps;
        *gmax_out = g;
    }
}

// gamma_r = max_j |sum_k B[r][k] Ai[k][j]|, accumulated as an atomic max of the bit pattern.
template <class T>
__global__ void __launch_bounds__(256) k_grade(int n, int m, const T* __restrict__ B, int ldb,
                                               const T* __restrict__ Ai, unsigned long long* gbits) {
    __shared__ T sb[16][64 + 1];
    __shared__ T sa[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < m; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, rr = e % 64;
            const int r = row0 + rr, k = k0 + kk;
            sb[kk][rr] = (r < n && k < m) ? B[(size_t)r * ldb + k] : T(0);
            const int c = col0 + rr;
            sa[kk][rr] = (c < m && k < m) ? Ai[(size_t)k * m + c] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T bv[4], av[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) bv[a] = sb[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) av[b] = sa[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += bv[a] * av[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        double mx = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (col0 + tx * 4 + b < m) {
                // a NaN entry counts as an infinite grade (fmax would drop it and report a row
                // of NaN as interpolating)
                const double v = fabs((double)acc[a][b]);
                mx = fmax(mx, v != v ? (double)INFINITY : v);
            }
        // combine the 16 threads that share this row (consecutive lanes)
        for (int o = 8; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o, 16));
        const int r = row0 + ty * 4 + a;
        if (tx == 0 && r < n) atomicMax(&gbits[r], (unsigned long long)__double_as_longlong(mx));
    }
}

__global__ void __launch_bounds__(kMvThreads) k_invert(int m, const double* A, double* Ai, double* W, int* status) {
    __shared__ ArgMax sbuf[33];
    __shared__ int s_flag;
    if (!gauss_jordan(A, Ai, W, m, sbuf, &s_flag) && threadIdx.x == 0) *status = kErrSingular;
}

}  // namespace

// The launchers return the number of kernels launched, or -1 if the launch itself failed (the
// error is taken off cudaGetLastError, so the caller reports it instead of reading stale results).
int launch_invert(int m, const double* A, double* Ai, double* W, int* status, cudaStream_t st) {
    k_invert<<<1, kMvThreads, 0, st>>>(m, A, Ai, W, status);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_maxvol(int n, int m, const double* B, double* Bs, double* D, double* W, int* perm, int* sel, double* A,
                  double* Ai, double* C, double tol, int max_iter, int* status, int* swaps, double* gmax,
                  cudaStream_t st, int start_given) {
    k_maxvol<<<1, kMvThreads, 0, st>>>(n, m, B, Bs, D, W, perm, sel, A, Ai, C, tol, max_iter, status, swaps, gmax,
                                       start_given);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_gather_columns(int rows, int w_in, const double* in, int w_out, const int* cols, double* out) {
    const size_t total = (size_t)rows * w_out;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / w_out, q = e - r * w_out;
        out[e] = in[r * w_in + cols[q]];
    }
}

int launch_gather_columns(int rows, int w_in, const double* in, int w_out, const int* cols, double* out,
                          cudaStream_t st) {
    const size_t total = (size_t)rows * w_out;
    if (total == 0) return 0;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
    k_gather_columns<<<blocks, 256, 0, st>>>(rows, w_in, in, w_out, cols, out);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <class T>
int launch_grade(int n, int m, const T* B, int ldb, const T* Ai, unsigned long long* gbits, cudaStream_t st) {
    if (n <= 0) return 0;
    cudaMemsetAsync(gbits, 0, sizeof(unsigned long long) * (size_t)n, st);
    dim3 grid((m + 63) / 64, (n + 63) / 64);
    k_grade<T><<<grid, 256, 0, st>>>(n, m, B, ldb, Ai, gbits);
    return 1;
}
template int launch_grade<float>(int, int, const float*, int, const float*, unsigned long long*, cudaStream_t);
template int launch_grade<double>(int, int, const double*, int, const double*, unsigned long long*, cudaStream_t);

}  // namespace mtp

// ------------------------------------------------------------------------------------------------
// Active-set selection without any allocation (mtp_select_active_set_noalloc in include/mtp.h).
//
// Some callers cannot let a library allocate device memory: a simulation loop that checks the
// extrapolation grade inside its time step must not pay for cudaMalloc (which may synchronise the
// whole device and stall the other streams), and applications that hand all device memory to
// their own pool allocator have nothing left for a library to take.  This entry point therefore
// runs the same MaxVol kernel with all of its scratch in one fixed array compiled into the library.
// Every GPU that loads the library holds this array (kNoAllocScratchDoubles doubles, 4 MiB) until
// the process exits.  Calls share it and it keeps the last call's contents, so calls that overlap
// on the GPU (two streams, or two host threads) race; the status word is cleared at every call.
// ------------------------------------------------------------------------------------------------
namespace mtp {
namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 19;  // 4 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace mtp

extern "C" mtp_status mtp_select_active_set_noalloc(int n_rows, int m, const double* b_rows, int32_t* selected,
                                                    double* a_inv, int* n_swaps, void* stream) {
    using namespace mtp;
    if (m < 1 || n_rows < m || !b_rows || !selected) return MTP_EINVAL;
    // layout inside the fixed array (in doubles): Bs, C [n m]; W [max(n m, 2 m m) + 2 m + n];
    // D [m]; A, A^-1 [m m]; then ints: perm [n], sel [m], status, swaps; then gmax.
    const size_t nm = (size_t)n_rows * m, mm = (size_t)m * m;
    const size_t w = (nm > 2 * mm ? nm : 2 * mm) + 2 * (size_t)m + n_rows;
    const size_t ints = (size_t)n_rows + m + 2;
    const size_t need = 2 * nm + w + m + 2 * mm + (ints + 1) / 2 + 1;
    if (need > kNoAllocScratchDoubles) return MTP_EINVAL;  // larger than the fixed scratch array
    double* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return MTP_ECUDA;
    double* Bs = base;
    double* C = Bs + nm;
    double* W = C + nm;
    double* D = W + w;
    double* A = D + m;
    double* Ai = A + mm;
    int* perm = reinterpret_cast<int*>(Ai + mm);
    int* sel = perm + n_rows;
    int* status = sel + m;
    int* swaps = status + 1;
    double* gmax = reinterpret_cast<double*>(base + (need - 1));
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, 2 * sizeof(int), st) != cudaSuccess) return MTP_ECUDA;
    if (launch_maxvol(n_rows, m, b_rows, Bs, D, W, perm, sel, A, Ai, C, 1e-3, 100 * m, status, swaps, gmax, st, 0) < 0)
        return MTP_ECUDA;
    int h[2] = {0, 0};
    if (cudaMemcpyAsync(h, status, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return MTP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MTP_ECUDA;
    if (h[0] & kErrSingular) return MTP_ESINGULAR;
    if (h[0] & kErrTimeout) return MTP_ETIMEOUT;
    if (cudaMemcpyAsync(selected, sel, sizeof(int) * m, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return MTP_ECUDA;
    if (a_inv && cudaMemcpyAsync(a_inv, Ai, sizeof(double) * mm, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MTP_ECUDA;
    if (n_swaps) *n_swaps = h[1];
    return cudaStreamSynchronize(st) == cudaSuccess ? MTP_OK : MTP_ECUDA;
}
