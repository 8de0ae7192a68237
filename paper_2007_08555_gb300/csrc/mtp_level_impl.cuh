// Kernels of one lev_max, instantiated by a generated translation unit that first includes the
// generated header and defines MTP_GEN_NS (its namespace) and MTP_LEVEL_FN (registry function).
//
// One evaluation (Sec. 2.1, Eqs. 1-4) runs four kernels:
//   k_moments   thread group per atom: radial functions f_mu (Eq. 3 with the Chebyshev basis of
//               Eq. 4) and the symmetric moment components M_{mu,nu}[a,b,c] = sum_j f_mu x^a y^b z^c,
//               accumulated in registers slice by slice (the slices are generated, unrolled code);
//   k_contract  warp per atom: the generated contraction program (every basis function B_alpha),
//               the site energy V_i = sum xi_alpha B_alpha (Eq. 2), then the adjoint program
//               dV_i/dM, all in shared memory;
//   k_pairgrad  thread group per atom: dV_i/dr_ij = sum adj * d(f_mu(r) mono(r))/dr per pair;
//   k_gather    thread per atom: F_i = sum_p (g_ip - g_{j_p, reverse}) and the virial
//               W = -sum g_ij (x) r_ij, reduced per configuration in double precision.
#include "mtp_common.cuh"
#include "mtp_level.h"

namespace mtp {
namespace MTP_GEN_NS {

using G = ::MTP_GEN_NS::Traits;

template <class T, int S>
struct SliceSel;
template <int S>
struct SliceSel<float, S> {
    using type = typename G::template F32<S>;
};
template <int S>
struct SliceSel<double, S> {
    using type = typename G::template F64<S>;
};
template <class T>
struct NumSlices;
template <>
struct NumSlices<float> {
    static constexpr int value = G::NS32_;
};
template <>
struct NumSlices<double> {
    static constexpr int value = G::NS64_;
};

__device__ __forceinline__ int clamp_species(int z, int S) { return z < 0 ? 0 : (z >= S ? S - 1 : z); }
__device__ __forceinline__ float my_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double my_sqrt(double x) { return sqrt(x); }

// f_mu(r) = (R_cut - r)^2 sum_b c_b T_b(x) and its r-derivative (Eqs. 3-4); Chebyshev T_b by the
// three-term recurrence, dT_b/dx by its derivative.  cz points at c[z_i][z_j][0][0].
template <class T, bool WANT_D>
__device__ __forceinline__ void radial(const T r, const T* __restrict__ cz, const int NQ, const T rmin,
                                       const T rcut, const T inv_span, T* f, T* df) {
    constexpr int NMU = G::NMU_;
    const T x = (T(2) * r - rmin - rcut) * inv_span;
    T F[NMU], D[NMU];
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
        F[mu] = cz[mu * NQ];
        D[mu] = T(0);
    }
    if (NQ > 1) {
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
            F[mu] += cz[mu * NQ + 1] * x;
            if (WANT_D) D[mu] += cz[mu * NQ + 1];
        }
    }
    T t0 = T(1), t1 = x, d0 = T(0), d1 = T(1);
    for (int b = 2; b < NQ; ++b) {
        const T t2 = T(2) * x * t1 - t0;
        const T d2 = T(2) * t1 + T(2) * x * d1 - d0;
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
            const T cb = cz[mu * NQ + b];
            F[mu] += cb * t2;
            if (WANT_D) D[mu] += cb * d2;
        }
        t0 = t1;
        t1 = t2;
        d0 = d1;
        d1 = d2;
    }
    const T u = rcut - r;
    const T u2 = u * u;
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
        f[mu] = F[mu] * u2;
        if (WANT_D) df[mu] = D[mu] * (T(2) * inv_span) * u2 - T(2) * F[mu] * u;
    }
}

template <class T>
__device__ __forceinline__ void load_c(const EvalCtx<T>& a, T* cs) {
    const int nc = a.S * a.S * G::NMU_ * a.NQ;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) cs[k] = a.c[k];
    __syncthreads();
}

// ----------------------------------------------------------------------------------------------
// k_moments
// ----------------------------------------------------------------------------------------------
template <class T, int S, int TPA>
__device__ __forceinline__ void moments_slice(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                              const T* cs) {
    using SL = typename SliceSel<T, S>::type;
    T acc[SL::SIZE];
#pragma unroll
    for (int t = 0; t < SL::SIZE; ++t) acc[t] = T(0);
    const size_t n = (size_t)a.n_atoms;
    if (active) {
        const int csz = G::NMU_ * a.NQ;
        for (int p = sub; p < cnt; p += TPA) {
            const size_t idx = (size_t)p * n + i;
            const int zj = a.jz[idx] >> 24;
            const T x = a.rx[idx], y = a.ry[idx], z = a.rz[idx];
            const T r = my_sqrt(x * x + y * y + z * z);
            T f[G::NMU_];
            radial<T, false>(r, cs + (zi * a.S + zj) * csz, a.NQ, a.rmin, a.rcut, a.inv_span, f, nullptr);
            SL::template mom<T>(x, y, z, f, acc);
        }
    }
    if (TPA > 1) {
#pragma unroll
        for (int t = 0; t < SL::SIZE; ++t) {
#pragma unroll
            for (int o = 1; o < TPA; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        }
    }
    if (active) {
        // the group's lanes store disjoint parts of the slice (tile layout [tile][C][32])
        T* dst = a.mom + (size_t)(i >> 5) * G::C_ * 32 + (i & 31);
#pragma unroll
        for (int t = 0; t < SL::SIZE; ++t)
            if (t % TPA == sub) dst[(size_t)(SL::BEGIN + t) * 32] = acc[t];
    }
}

template <class T, int S, int NS, int TPA>
__device__ __forceinline__ void moments_all(const EvalCtx<T>& a, int i, int sub, bool active, int zi, int cnt,
                                            const T* cs) {
    if constexpr (S < NS) {
        moments_slice<T, S, TPA>(a, i, sub, active, zi, cnt, cs);
        moments_all<T, S + 1, NS, TPA>(a, i, sub, active, zi, cnt, cs);
    }
}

template <class T, int TPA>
__global__ void __launch_bounds__(128) k_moments(const EvalCtx<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cs = reinterpret_cast<T*>(smem_raw);
    load_c(a, cs);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    const int n_groups = ((a.n_atoms + 31) / 32) * 32;  // whole warps stay converged for the shuffles
    for (int g = gtid; g < n_groups * TPA; g += stride) {
        const int i = g / TPA, sub = g % TPA;
        const bool active = i < a.n_atoms;
        int zi = 0, cnt = 0;
        if (active) {
            zi = clamp_species(a.types[i], a.S);  // out-of-range species are reported by the neighbour build
            cnt = a.count[i];
        }
        moments_all<T, 0, NumSlices<T>::value, TPA>(a, i, sub, active, zi, cnt, cs);
    }
}

// ----------------------------------------------------------------------------------------------
// k_contract: warp per atom
// ----------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void run_forward(const EvalCtx<T>& a, T* val, int lane) {
    int row = 0;
    for (int l = 0; l < a.fwd_layers; ++l) {
        const int end = a.fwd_layer_end[l];
        T acc = T(0);
        for (; row < end; ++row) {
            const unsigned ij = a.fwd_ij[row * 32 + lane];
            const unsigned kf = a.fwd_kf[row * 32 + lane];
            const unsigned fl = kf >> 16;
            if (!(fl & 4u)) {
                if (fl & 1u) acc = T(0);
                acc += T(a.fwd_w[row * 32 + lane]) * val[ij & 0xffffu] * val[ij >> 16];
                if (fl & 2u) val[kf & 0xffffu] = acc;
            }
        }
        __syncwarp();
    }
}

template <class T>
__device__ __forceinline__ void run_adjoint(const EvalCtx<T>& a, const T* val, T* adj, int lane) {
    int row = 0;
    for (int l = 0; l < a.adj_layers; ++l) {
        const int end = a.adj_layer_end[l];
        T acc = T(0);
        for (; row < end; ++row) {
            const unsigned ij = a.adj_ij[row * 32 + lane];
            const unsigned kf = a.adj_kf[row * 32 + lane];
            const unsigned fl = kf >> 16;
            if (!(fl & 4u)) {
                const unsigned k = kf & 0xffffu;
                if (fl & 1u) acc = adj[k];
                acc += T(a.adj_w[row * 32 + lane]) * val[ij & 0xffffu] * adj[ij >> 16];
                if (fl & 2u) adj[k] = acc;
            }
        }
        __syncwarp();
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_contract(const EvalCtx<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int V = G::V_, C = G::C_, M = G::M_;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    T* seed = reinterpret_cast<T*>(smem_raw);
    T* val = seed + V + warp * 2 * V;
    T* adj = val + V;
    for (int v = threadIdx.x; v < V; v += blockDim.x) seed[v] = a.seed[v];
    __syncthreads();
    double esum = 0.0;
    int ecfg = -1;
    const int total_warps = gridDim.x * wpb;
    for (int i = blockIdx.x * wpb + warp; i < a.n_atoms; i += total_warps) {
        const T* msrc = a.mom + (size_t)(i >> 5) * C * 32 + (i & 31);
        for (int c = lane; c < C; c += 32) val[c] = msrc[(size_t)c * 32];
        __syncwarp();
        run_forward(a, val, lane);
        // site energy and basis values
        const int cfg = a.cfg_of[i];
        T e = T(0);
        for (int al = lane; al < M; al += 32) {
            const T b = val[a.basis_value[al]];
            e += a.xi[al] * b;
            if (a.b_atoms) a.b_atoms[(size_t)i * M + al] = (double)b;
            if (a.b_rows) atomicAdd(&a.b_rows[(size_t)cfg * M + al], (double)b);
        }
        const double ed = warp_sum((double)e);
        if (lane == 0) {
            if (a.site) a.site[i] = ed;
            if (cfg != ecfg) {
                if (ecfg >= 0 && a.energy) atomicAdd(&a.energy[ecfg], esum);
                ecfg = cfg;
                esum = 0.0;
            }
            esum += ed;
        }
        // adjoint: dV/dval seeded with xi at the basis values
        for (int v = lane; v < V; v += 32) adj[v] = seed[v];
        __syncwarp();
        run_adjoint(a, val, adj, lane);
        T* adst = a.adjm + (size_t)(i >> 5) * C * 32 + (i & 31);
        for (int c = lane; c < C; c += 32) adst[(size_t)c * 32] = adj[c];
        __syncwarp();
    }
    if (lane == 0 && ecfg >= 0 && a.energy) atomicAdd(&a.energy[ecfg], esum);
}

// ----------------------------------------------------------------------------------------------
// k_pairgrad: g_ij = dV_i/dr_ij
// ----------------------------------------------------------------------------------------------
template <class T, int S, int TPA>
__device__ __forceinline__ void pairgrad_slice(const EvalCtx<T>& a, int i, int sub, int zi, int cnt, const T* cs) {
    using SL = typename SliceSel<T, S>::type;
    T adjs[SL::SIZE];
    const T* src = a.adjm + (size_t)(i >> 5) * G::C_ * 32 + (i & 31);
#pragma unroll
    for (int t = 0; t < SL::SIZE; ++t) adjs[t] = src[(size_t)(SL::BEGIN + t) * 32];
    const size_t n = (size_t)a.n_atoms;
    const int csz = G::NMU_ * a.NQ;
    for (int p = sub; p < cnt; p += TPA) {
        const size_t idx = (size_t)p * n + i;
        const int zj = a.jz[idx] >> 24;
        const T x = a.rx[idx], y = a.ry[idx], z = a.rz[idx];
        const T r = my_sqrt(x * x + y * y + z * z);
        T f[G::NMU_], df[G::NMU_];
        radial<T, true>(r, cs + (zi * a.S + zj) * csz, a.NQ, a.rmin, a.rcut, a.inv_span, f, df);
        T s = T(0), gx = T(0), gy = T(0), gz = T(0);
        SL::template grad<T>(x, y, z, f, df, adjs, s, gx, gy, gz);
        const T sr = s / r;
        gx += sr * x;
        gy += sr * y;
        gz += sr * z;
        if (S == 0) {
            a.gx[idx] = gx;
            a.gy[idx] = gy;
            a.gz[idx] = gz;
        } else {
            a.gx[idx] += gx;
            a.gy[idx] += gy;
            a.gz[idx] += gz;
        }
    }
}

template <class T, int S, int NS, int TPA>
__device__ __forceinline__ void pairgrad_all(const EvalCtx<T>& a, int i, int sub, int zi, int cnt, const T* cs) {
    if constexpr (S < NS) {
        pairgrad_slice<T, S, TPA>(a, i, sub, zi, cnt, cs);
        pairgrad_all<T, S + 1, NS, TPA>(a, i, sub, zi, cnt, cs);
    }
}

template <class T, int TPA>
__global__ void __launch_bounds__(128) k_pairgrad(const EvalCtx<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cs = reinterpret_cast<T*>(smem_raw);
    load_c(a, cs);
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int g = gtid; g < a.n_atoms * TPA; g += stride) {
        const int i = g / TPA, sub = g % TPA;
        pairgrad_all<T, 0, NumSlices<T>::value, TPA>(a, i, sub, clamp_species(a.types[i], a.S), a.count[i], cs);
    }
}

// ----------------------------------------------------------------------------------------------
// k_gather: forces and virial
// ----------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128) k_gather(const EvalCtx<T> a) {
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const size_t n = (size_t)a.n_atoms;
    const int n_round = ((a.n_atoms + 31) / 32) * 32;
    for (int i = i0; i < n_round; i += stride) {
        const bool active = i < a.n_atoms;
        T F[3] = {T(0), T(0), T(0)};
        T W[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) W[k] = T(0);
        int cfg = -1;
        if (active) {
            cfg = a.cfg_of[i];
            const int cnt = a.count[i];
            for (int p = 0; p < cnt; ++p) {
                const size_t idx = (size_t)p * n + i;
                const T g[3] = {a.gx[idx], a.gy[idx], a.gz[idx]};
                const T r[3] = {a.rx[idx], a.ry[idx], a.rz[idx]};
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    F[u] += g[u];
#pragma unroll
                    for (int v = 0; v < 3; ++v) W[3 * u + v] -= g[u] * r[v];
                }
                const int q = a.rev[idx];
                if (q >= 0) {
                    const size_t ridx = (size_t)q * n + (a.jz[idx] & 0xffffff);
                    F[0] -= a.gx[ridx];
                    F[1] -= a.gy[ridx];
                    F[2] -= a.gz[ridx];
                }
            }
            if (a.forces) {
                a.forces[3 * (size_t)i + 0] = (double)F[0];
                a.forces[3 * (size_t)i + 1] = (double)F[1];
                a.forces[3 * (size_t)i + 2] = (double)F[2];
            }
        }
        if (!a.virial) continue;
        // per-configuration reduction: one atomic per warp when the warp lies in one configuration
        const int c0 = __shfl_sync(0xffffffffu, cfg, 0);
        const bool uniform = __all_sync(0xffffffffu, cfg == c0 || cfg < 0);
        if (uniform) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const double s = warp_sum((double)W[k]);
                if (lane == 0 && c0 >= 0) atomicAdd(&a.virial[(size_t)c0 * 9 + k], s);
            }
        } else if (active) {
#pragma unroll
            for (int k = 0; k < 9; ++k) atomicAdd(&a.virial[(size_t)cfg * 9 + k], (double)W[k]);
        }
    }
}

// ----------------------------------------------------------------------------------------------
// launcher
// ----------------------------------------------------------------------------------------------
template <class T, int TPA>
int launch_pairs(const EvalCtx<T>& a, cudaStream_t st, int n_sm, bool moments) {
    const int threads = 128;
    const size_t cbytes = sizeof(T) * (size_t)a.S * a.S * G::NMU_ * a.NQ;
    const long work = (long)(((a.n_atoms + 31) / 32) * 32) * TPA;
    int blocks = (int)((work + threads - 1) / threads);
    const int max_blocks = n_sm * 16;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (moments)
        k_moments<T, TPA><<<blocks, threads, cbytes, st>>>(a);
    else
        k_pairgrad<T, TPA><<<blocks, threads, cbytes, st>>>(a);
    return 1;
}

template <class T>
int launch_pairs_tpa(const EvalCtx<T>& a, cudaStream_t st, int n_sm, bool moments) {
    switch (a.tpa) {
        case 8: return launch_pairs<T, 8>(a, st, n_sm, moments);
        case 4: return launch_pairs<T, 4>(a, st, n_sm, moments);
        case 2: return launch_pairs<T, 2>(a, st, n_sm, moments);
        default: return launch_pairs<T, 1>(a, st, n_sm, moments);
    }
}

template <class T>
int eval_all(const EvalCtx<T>& a, cudaStream_t st, int n_sm, cudaEvent_t* marks) {
    if (a.n_atoms == 0) return 0;
    int launches = 0;
    if (marks) cudaEventRecord(marks[kPhaseMoments], st);
    launches += launch_pairs_tpa<T>(a, st, n_sm, true);
    if (marks) cudaEventRecord(marks[kPhaseContract], st);
    {
        const int threads = 256;
        const int wpb = threads / 32;
        const size_t smem = sizeof(T) * (size_t)G::V_ * (1 + 2 * wpb);
        if (smem > 200 * 1024) return -1000;  // not reachable for lev_max <= 20
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_contract<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set = true;
        }
        int blocks = (a.n_atoms + wpb - 1) / wpb;
        int per_sm = (int)((200 * 1024) / (smem ? smem : 1));
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 4) per_sm = 4;
        if (blocks > n_sm * per_sm * 4) blocks = n_sm * per_sm * 4;
        k_contract<T><<<blocks, threads, smem, st>>>(a);
        ++launches;
    }
    if (marks) cudaEventRecord(marks[kPhasePairgrad], st);
    launches += launch_pairs_tpa<T>(a, st, n_sm, false);
    if (marks) cudaEventRecord(marks[kPhaseGather], st);
    {
        const int threads = 128;
        int blocks = (a.n_atoms + threads - 1) / threads;
        if (blocks > n_sm * 16) blocks = n_sm * 16;
        k_gather<T><<<blocks, threads, 0, st>>>(a);
        ++launches;
    }
    if (marks) cudaEventRecord(marks[kPhases], st);
    return launches;
}

int eval_f32(const EvalCtx<float>& a, cudaStream_t st, int n_sm, cudaEvent_t* marks) {
    return eval_all<float>(a, st, n_sm, marks);
}
int eval_f64(const EvalCtx<double>& a, cudaStream_t st, int n_sm, cudaEvent_t* marks) {
    return eval_all<double>(a, st, n_sm, marks);
}

}  // namespace MTP_GEN_NS

const LevelOps* MTP_LEVEL_FN() {
    namespace g = ::MTP_GEN_NS;
    static const LevelOps ops = {
        g::L, g::C, g::V, g::M, g::NMU, g::NUMAX,
        g::level_table, g::LEVEL_TABLE_LEN, g::basis_value,
        g::fwd_ij, g::fwd_kf, g::fwd_w, g::fwd_layer_rows, g::FWD_ROWS, g::FWD_LAYERS,
        g::adj_ij, g::adj_kf, g::adj_w, g::adj_layer_rows, g::ADJ_ROWS, g::ADJ_LAYERS,
        g::PROGRAM_OPS, g::FLOP_PAIR_MOMENTS, g::FLOP_PAIR_ADJOINT, g::FLOP_ATOM_PROGRAM,
        &MTP_GEN_NS::eval_f32, &MTP_GEN_NS::eval_f64};
    return &ops;
}

}  // namespace mtp
